// vi.cuh -- Voronoi initialisation of tonal optimisation (Sec. 5.3).
//
// The mask values are moved towards interpolating local averages of f: the
// modified Richardson iteration
//     g <- g + tau C W (f - u),   u = A^{-1} C g (one inpainting per step),
// started from g = f on the mask and stopped at the first step that raises
// the MSE of u (the previous g is kept). Row s of W averages over the
// influence zone of mask pixel s:
//   mode 0  its Voronoi cell (exact labels, as in densification), weight
//           1 / (1 + ln(1 + d)), d = distance to s;
//   mode 1  its Voronoi cell, constant weight;
//   mode 2  its 3x3 neighbourhood clipped to the image (error balancing of
//           Galic et al.), constant weight.
// Modes 0 and 1 accumulate w (f - u) of every pixel into its site with
// integer atomics on values scaled by 2^32 (order-independent, so the result
// does not depend on the schedule); the weights' sums per site are formed the
// same way once per call.
#pragma once
#include "common.cuh"
#include "stencil.cuh"
#include "solver.h"
#include "densify.cuh"   // exact Voronoi labels (k_vor_columns, k_vor_rows)

constexpr int kViThreads = 256;
constexpr float kViScalef = 4294967296.f;   // 2^32

// Weight of every pixel of the zone of its Voronoi site V[p] (modes 0, 1)
// and the per-site weight sums.
__global__ void __launch_bounds__(kViThreads) k_vi_weights(const int* __restrict__ V, int H, int W, int mode,
                                                           float* __restrict__ w,
                                                           unsigned long long* __restrict__ den) {
    const int x = blockIdx.x * kViThreads + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const size_t p = (size_t)y * W + x;
    const int s = V[p];
    float wv = 1.f;
    if (mode == 0) {
        const int sy = s / W, sx = s - sy * W;
        const float dx = (float)(x - sx), dy = (float)(y - sy);
        const float d = sqrtf(dx * dx + dy * dy);
        wv = 1.f / (1.f + log1pf(d));
    }
    w[p] = wv;
    atomicAdd(den + s, (unsigned long long)llrintf(wv * kViScalef));
}

// Per channel: sum of (f - u)^2 over the image into `red`; with V != nullptr
// also num[ch][V[p]] += w_p (f_p - u_p) (scaled integers).
__global__ void __launch_bounds__(kViThreads) k_vi_accum(LevelArr F, DFc f, DFc u, const int* __restrict__ V,
                                                         const float* __restrict__ w,
                                                         unsigned long long* __restrict__ num, GridReduce red) {
    const int ch = blockIdx.y;
    const size_t co = (size_t)ch * F.cs;
    const size_t N = (size_t)F.H * F.W;
    float s2 = 0.f;
    for (int y = blockIdx.x; y < F.H; y += gridDim.x) {
        const size_t ro = co + (size_t)y * F.pitch;
        for (int x = threadIdx.x; x < F.W; x += kViThreads) {
            const size_t i = ro + x;
            const float e = (f.hi[i] - u.hi[i]) + (f.lo[i] - u.lo[i]);
            s2 = fmaf(e, e, s2);
            if (V) {
                const size_t p = (size_t)y * F.W + x;
                // scaling by a power of two is exact; the rounding to an
                // integer drops only bits below 2^-32
                atomicAdd(num + (size_t)ch * N + V[p], (unsigned long long)llrintf((w[p] * e) * kViScalef));
            }
        }
    }
    const double tot = (double)block_sum_f(s2);
    grid_reduce_commit(red, ch, blockIdx.x, tot);
}

// g += tau * num / den at the mask pixels (modes 0, 1); num is cleared for
// the next accumulation.
__global__ void __launch_bounds__(kViThreads) k_vi_update(LevelArr F, MaskView m, unsigned long long* __restrict__ num,
                                                          const unsigned long long* __restrict__ den, DF g,
                                                          double tau) {
    const int ch = blockIdx.y;
    const MaskView mc = m.ch(ch);
    const size_t N = (size_t)F.H * F.W;
    for (int y = blockIdx.x; y < F.H; y += gridDim.x) {
        for (int x = threadIdx.x; x < F.W; x += kViThreads) {
            if (!mc.known(x, y)) continue;
            const size_t p = (size_t)y * F.W + x;
            const size_t q = (size_t)ch * N + p;
            const double r = (double)(long long)num[q] / (double)den[p];
            num[q] = 0ull;
            const size_t i = (size_t)ch * F.cs + (size_t)y * F.pitch + x;
            float th, tl;
            df_from_d(tau * r, th, tl);
            float h, l;
            df_add(g.hi[i], g.lo[i], th, tl, h, l);
            g.hi[i] = h;
            g.lo[i] = l;
        }
    }
}

// Mode 2: g += tau * mean over the clipped 3x3 neighbourhood of (f - u) at
// the mask pixels.
__global__ void __launch_bounds__(kViThreads) k_vi_neigh(LevelArr F, MaskView m, DFc f, DFc u, DF g, double tau) {
    const int ch = blockIdx.y;
    const MaskView mc = m.ch(ch);
    const size_t co = (size_t)ch * F.cs;
    for (int y = blockIdx.x; y < F.H; y += gridDim.x) {
        for (int x = threadIdx.x; x < F.W; x += kViThreads) {
            if (!mc.known(x, y)) continue;
            double acc = 0.0;
            int n = 0;
            for (int yy = max(y - 1, 0); yy <= min(y + 1, F.H - 1); ++yy)
                for (int xx = max(x - 1, 0); xx <= min(x + 1, F.W - 1); ++xx) {
                    const size_t j = co + (size_t)yy * F.pitch + xx;
                    acc += (double)((f.hi[j] - u.hi[j]) + (f.lo[j] - u.lo[j]));
                    ++n;
                }
            const size_t i = co + (size_t)y * F.pitch + x;
            float th, tl;
            df_from_d(tau * acc / n, th, tl);
            float h, l;
            df_add(g.hi[i], g.lo[i], th, tl, h, l);
            g.hi[i] = h;
            g.lo[i] = l;
        }
    }
}

// The Voronoi initialisation on the context's G (level-0 layout, f on the
// mask or the caller's g0 on entry). Returns the number of accepted steps,
// the MSE of the kept iterate and, when it is still at hand, its inpainting
// (*u_kept; hi == nullptr after a rejected last step). Uses the inpainting
// buffers U0/U1 and P as the backup of G.
int Ctx::tonal_vi(int& steps, double& mse_best, DF* u_kept) {
    int rc;
    steps = 0;
    u_kept->hi = u_kept->lo = nullptr;
    const int mode = (int)(p.vi_weight + 0.5);
    const double tau = p.vi_tau;
    const int max_it = (int)p.vi_max_iter;
    const size_t N = (size_t)H * W;
    const DF G = dfv[kG];
    const DF Gb = dfv[kP];
    const size_t gbytes = (size_t)nch * lev[0].cs * 8;   // hi and lo halves, contiguous
    int* V = nullptr;
    float* wgt = nullptr;
    unsigned long long* den = nullptr;
    unsigned long long* num = nullptr;
    if (mode != 2) {
        size_t bytes = 0;
        auto acc = [&](size_t b) { bytes += (b + 255) & ~(size_t)255; };
        acc(N * 4);                 // ys
        acc(N * 4);                 // V
        acc(N * 4);                 // weights
        acc(N * 8);                 // per-site weight sums
        acc((size_t)nch * N * 8);   // per-site weighted error sums
        if ((rc = vws.reserve(*this, std::max(vws.cap, bytes), "Voronoi initialisation workspace"))) return rc;
        int* ys = (int*)vws.take(N * 4);
        V = (int*)vws.take(N * 4);
        wgt = (float*)vws.take(N * 4);
        den = (unsigned long long*)vws.take(N * 8);
        num = (unsigned long long*)vws.take((size_t)nch * N * 8);
        const MaskView mv = mview(0);
        launch_vor_columns(mv, ys, stream);
        k_vor_rows<<<dim3((W + 127) / 128, H), 128, 0, stream>>>(ys, H, W, V);
        cudaMemsetAsync(den, 0, N * 8, stream);
        cudaMemsetAsync(num, 0, (size_t)nch * N * 8, stream);
        k_vi_weights<<<dim3((W + kViThreads - 1) / kViThreads, H), kViThreads, 0, stream>>>(V, H, W, mode, wgt, den);
        launches += 3;
    }
    const int parts = std::min(maxparts_, 4 * 148);
    const dim3 vgrid(parts, nch);
    const DFc F = cview(dfv[kF]);
    SolveSpec su;
    su.u[0] = dfv[kU0];
    su.u[1] = dfv[kU1];
    su.cur = 0;
    su.rhs = RHS_DATA;
    su.d = cview(G);
    su.start = START_FMG;
    su.tol = p.vi_inner_tol;
    su.max_iter = (int)p.max_vcycles;
    double e2[kMaxCh];
    auto inpaint_and_measure = [&](double& mse) -> int {
        int r = solve(su);
        if (r != HDI_OK && r != HDI_ERR_NOT_CONVERGED) return fail(r, "Voronoi initialisation: inpainting: %s", err.c_str());
        su.start = START_WARM;
        k_vi_accum<<<vgrid, kViThreads, 0, stream>>>(arr(0), F, cview(su.u[su.cur]), V, wgt, num,
                                                      reducer(kSlotViE, parts));
        ++launches;
        if ((r = read_slot(kSlotViE, e2))) return r;
        double s = 0.0;
        for (int c = 0; c < nch; ++c) s += e2[c];
        if (!std::isfinite(s)) return fail(HDI_ERR_NONFINITE, "Voronoi initialisation: non-finite error");
        mse = s / ((double)nch * N);
        return HDI_OK;
    };
    if ((rc = inpaint_and_measure(mse_best))) return rc;
    for (int k = 0; k < max_it; ++k) {
        cudaMemcpyAsync(Gb.hi, G.hi, gbytes, cudaMemcpyDeviceToDevice, stream);
        if (mode == 2)
            k_vi_neigh<<<vgrid, kViThreads, 0, stream>>>(arr(0), mview(0), F, cview(su.u[su.cur]), G, tau);
        else
            k_vi_update<<<vgrid, kViThreads, 0, stream>>>(arr(0), mview(0), num, den, G, tau);
        ++launches;
        double mse = 0.0;
        if ((rc = inpaint_and_measure(mse))) return rc;
        if (p.trace > 0) fprintf(stderr, "[hdi vi] step %d mse %.6f (best %.6f)\n", k, mse, mse_best);
        if (mse > mse_best) {
            cudaMemcpyAsync(G.hi, Gb.hi, gbytes, cudaMemcpyDeviceToDevice, stream);
            if (num) cudaMemsetAsync(num, 0, (size_t)nch * N * 8, stream);
            return cuda_check(cudaGetLastError(), "Voronoi initialisation");
        }
        mse_best = mse;
        ++steps;
    }
    *u_kept = su.u[su.cur];
    return cuda_check(cudaGetLastError(), "Voronoi initialisation");
}

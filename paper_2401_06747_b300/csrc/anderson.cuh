// anderson.cuh -- Anderson acceleration of the RAS fixed-point iteration.
//
// Alg. 2 is the stationary iteration g <- g + P r(g), with P the weighted
// sum of local solves and r(g) = B^T (f - B g) affine in g. Anderson
// acceleration (type II, window m) replaces the plain step by
//   g_{n+1} = g_n + f_n - (dX + dF) gamma,  gamma = argmin ||f_n - dF gamma||,
// where f_n = P r_n and the columns of dX, dF are the last m differences of
// iterates and of f. For an affine map this is a Krylov method over the
// same residuals, so it needs no operator application beyond the warm-started
// residual evaluations Alg. 2 already performs. All vectors live on the mask
// pixels only, in a compact raster-order list.
#pragma once
#include "common.cuh"
#include "stencil.cuh"

constexpr int kAAMax = 8;   // largest Anderson window
constexpr int kAAParts = 128;  // CTAs per channel of the dot-product kernel

// Ones per row (warp per row).
__global__ void k_row_counts(MaskView m, int* __restrict__ cnt) {
    const int y = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (y >= m.H) return;
    const int nw = (m.W + 31) / 32;
    int c = 0;
    for (int w = lane; w < nw; w += 32) c += __popc(m.bits[(size_t)y * m.wpitch + w]);
    c = __reduce_add_sync(HDI_FULL, c);
    if (lane == 0) cnt[y] = c;
}

// Compact list of known pixels, raster order: idx[rowoff[y] + k] = y*pitch + x.
__global__ void k_compact_fill(MaskView m, int pitch, const int* __restrict__ rowoff, int* __restrict__ idx) {
    const int y = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (y >= m.H) return;
    const int nw = (m.W + 31) / 32;
    int base = rowoff[y];
    for (int w0 = 0; w0 < nw; w0 += 32) {
        const int w = w0 + lane;
        uint32_t bits = (w < nw) ? m.bits[(size_t)y * m.wpitch + w] : 0u;
        const int c = __popc(bits);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(HDI_FULL, incl, o);
            if (lane >= o) incl += t;
        }
        int pos = base + incl - c;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            idx[pos++] = y * pitch + w * 32 + b;
        }
        base += __shfl_sync(HDI_FULL, incl, 31);
    }
}

struct AAArgs {
    int M;              // known pixels per channel
    long long cs;       // channel stride of the full-layout arrays
    int nch, k, slot, mwin;
    float beta;         // mixing: step = beta f_n - sum_j gamma_j (dX_j + beta dF_j)
    const int* idx;     // [M]
    const float* fvfull;// P r in full layout (valid on known pixels)
    float* fv;          // [nch][M] current f_n
    float* fvprev;      // [nch][M] f_{n-1}
    float* dF;          // [mwin][nch][M]
    float* dX;          // [mwin][nch][M]
    DF g;               // iterate (full layout)
    const double* gamma;// [nch][kAAMax]
    double* partials;   // dots: [nch][ndots][nparts]
    double* out;        // [nch][ndots]
    unsigned* ticket;
    int nparts;
};

// Gather f_n, form dF of the newest slot (f_n - f_{n-1}) when n >= 1, and the
// dot products dF_i . dF_j (i <= j) and dF_i . f_n of the active window, per
// channel, reduced deterministically. Grid: (nparts, nch), 256 threads.
template <int K>
__global__ void __launch_bounds__(256) k_aa_gather(AAArgs a, int new_slot) {
    const int ch = blockIdx.y;
    const int part = blockIdx.x;
    constexpr int ND = K * (K + 1) / 2 + K;
    constexpr int NA = ND > 0 ? ND : 1;
    // per-thread dot products as compensated FP32 sums (TwoSum on every term:
    // value as + ae, about twice the FP32 precision)
    float as[NA], ae[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) as[q] = ae[q] = 0.f;
    auto acc = [&](int q, float x) {
        const float t = as[q] + x;
        const float bp = t - as[q];
        ae[q] += (as[q] - (t - bp)) + (x - bp);
        as[q] = t;
    };
    const size_t co = (size_t)ch * a.M;
    const size_t vs = (size_t)a.nch * a.M;   // stride between window slots
    const int stride = a.nparts * 256;
    // U elements per thread and round: all their loads are issued before the
    // arithmetic (the kernel runs one or two CTAs per SM, so the load latency
    // is hidden by loads in flight rather than by resident warps). The
    // newest difference dF[slot] is formed here (f_n - f_{n-1}); the older
    // ones are read.
    constexpr int U = 4;
    constexpr int KD = K > 0 ? K : 1;
    for (int i0 = part * 256 + threadIdx.x; i0 < a.M; i0 += U * stride) {
        int ix[U];
        float f[U], fp[U], d[U][KD];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * stride;
            ix[u] = (i < a.M) ? a.idx[i] : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * stride;
            const bool ok = i < a.M;
            f[u] = ok ? a.fvfull[ch * a.cs + ix[u]] : 0.f;
            fp[u] = ok ? a.fvprev[co + i] : 0.f;
#pragma unroll
            for (int j = 1; j < K; ++j) {
                const int sl = (a.slot - j + a.mwin * 4) % a.mwin;
                d[u][j] = ok ? a.dF[(size_t)sl * vs + co + i] : 0.f;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * stride;
            if (i >= a.M) break;
            const float df = f[u] - fp[u];
            a.fv[co + i] = f[u];
            if (new_slot >= 0) a.dF[(size_t)new_slot * vs + co + i] = df;   // slot j = 0 of the window
            a.fvprev[co + i] = f[u];
            d[u][0] = df;
        }
        if (K > 0) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (i0 + u * stride >= a.M) break;
                int q = 0;
#pragma unroll
                for (int r = 0; r < K; ++r)
#pragma unroll
                    for (int c = r; c < K; ++c) acc(q++, d[u][r] * d[u][c]);
#pragma unroll
                for (int r = 0; r < K; ++r) acc(q++, d[u][r] * f[u]);
            }
        }
    }
    if constexpr (K == 0) {
        return;
    } else {
        // block reduce all dots at once: warp sums in FP64, one shared-memory
        // exchange, then thread q adds the warps' values of dot q
        __shared__ double wsum[8][NA];
#pragma unroll
        for (int q = 0; q < ND; ++q) {
            const double t = warp_sum_d((double)as[q] + (double)ae[q]);
            if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5][q] = t;
        }
        __syncthreads();
        if (threadIdx.x < ND) {
            double t = 0.0;
#pragma unroll
            for (int w = 0; w < 8; ++w) t += wsum[w][threadIdx.x];
            a.partials[((size_t)ch * ND + threadIdx.x) * a.nparts + part] = t;
            __threadfence();   // each writer publishes its partial before the ticket
        }
        __shared__ bool last;
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned t = atomicAdd(a.ticket, 1u);
            last = (t == (unsigned)(a.nparts * a.nch - 1));
        }
        __syncthreads();
        if (!last) return;
        __threadfence();
        // the last CTA sums the partials of every (channel, dot) pair, one warp
        // per pair (fixed order: lane-strided sums, then the warp tree), with no
        // block-wide barrier between pairs
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int j = warp; j < a.nch * ND; j += 8) {
            const double* src = a.partials + (size_t)j * a.nparts;   // [channel][dot] = j
            double s = 0.0;
            for (int p = lane; p < a.nparts; p += 32) s += __ldcg(src + p);
            s = warp_sum_d(s);
            if (lane == 0) a.out[j] = s;
        }
        if (threadIdx.x == 0) *a.ticket = 0u;
    }
}

// step = beta f_n - sum_j gamma_j (dX_j + beta dF_j);  g += step;  dX[write_slot] = step.
__global__ void __launch_bounds__(256) k_aa_update(AAArgs a, int write_slot) {
    const int ch = blockIdx.y;
    const size_t co = (size_t)ch * a.M;
    const size_t vs = (size_t)a.nch * a.M;
    for (int i = blockIdx.x * 256 + threadIdx.x; i < a.M; i += gridDim.x * 256) {
        float s = a.beta * a.fv[co + i];
        for (int j = 0; j < a.k; ++j) {
            const int sl = (a.slot - j + a.mwin * 4) % a.mwin;
            const float gj = (float)a.gamma[ch * kAAMax + j];
            s -= gj * fmaf(a.beta, a.dF[(size_t)sl * vs + co + i], a.dX[(size_t)sl * vs + co + i]);
        }
        const size_t p = ch * a.cs + a.idx[i];
        float h, l;
        df_add(a.g.hi[p], a.g.lo[p], s, 0.f, h, l);
        a.g.hi[p] = h;
        a.g.lo[p] = l;
        a.dX[(size_t)write_slot * vs + co + i] = s;
    }
}

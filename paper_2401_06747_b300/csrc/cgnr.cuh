// cgnr.cuh -- vector kernels of CGNR tonal optimisation (Sec. 5.1,
// "Improvements"): conjugate gradients on the normal equations
// B^T B g = B^T f, carried on the inpainting residual r = f - B g.
//
//   y = B g, z = B^T (f - y), p = z
//   repeat: w = B p (an inpainting with data p)
//           alpha = <z, p> / <w, w>;  y += alpha w;  g += alpha p
//           z = B^T (f - y) (adjoint solve + k_tonal_residual)
//           beta = <z, z> / <z_old, z_old>;  p = z + beta p
//
// y, g and p are double-float images of level-0 layout; z is the FP32 output
// of k_tonal_residual (valid on mask pixels). alpha and beta are formed per
// channel on the device from the FP64 reduction slots, so no host round trip
// sits between the steps. Each channel is its own least-squares problem.
#pragma once
#include "common.cuh"
#include "stencil.cuh"

constexpr int kCgnrThreads = 256;

// <w, w> over all pixels (w = B p, double-float) and <z, p> over the mask
// pixels, per channel. The kernels here walk the image row-cyclically: CTA x
// takes rows x, x + gridDim.x, ...
__global__ void __launch_bounds__(kCgnrThreads) k_cgnr_dots(LevelArr F, MaskView m, DFc w, const float* __restrict__ z,
                                                            DFc p, GridReduce red_ww, GridReduce red_zp) {
    const int ch = blockIdx.y;
    const MaskView mc = m.ch(ch);
    const size_t co = (size_t)ch * F.cs;
    float sw = 0.f, sz = 0.f;
    for (int y = blockIdx.x; y < F.H; y += gridDim.x) {
        const size_t ro = co + (size_t)y * F.pitch;
        for (int x = threadIdx.x; x < F.W; x += kCgnrThreads) {
            const float v = w.hi[ro + x] + w.lo[ro + x];
            sw = fmaf(v, v, sw);
            if (mc.known(x, y)) sz = fmaf(z[ro + x], p.hi[ro + x] + p.lo[ro + x], sz);
        }
    }
    const double tw = (double)block_sum_f(sw);
    grid_reduce_commit(red_ww, ch, blockIdx.x, tw);
    const double tz = (double)block_sum_f(sz);
    grid_reduce_commit(red_zp, ch, blockIdx.x, tz);
}

// (h, l) += a * (wh, wl) in double-float, a = (ah, al).
__device__ __forceinline__ void df_axpy(float ah, float al, float wh, float wl, float& h, float& l) {
    const float p = ah * wh;
    float e = fmaf(ah, wh, -p);              // exact error of the leading product
    e = fmaf(ah, wl, fmaf(al, wh, e));
    float sh, sl;
    fast_two_sum(p, e, sh, sl);
    df_add(h, l, sh, sl, h, l);
}

// y += alpha w on every pixel, g += alpha p on mask pixels, per channel
// alpha = <z, p> / <w, w>: the exact minimiser of ||f - B (g + t p)|| over t
// for the current z. In exact arithmetic <z, p> = <z, z> (z is orthogonal to
// the previous direction), the textbook step; with inexact inner solves
// that orthogonality is only approximate and the line-search form keeps
// every step a descent step. alpha = 0 where <w, w> = 0 or <z, p> <= 0.
// CTA (0, ch) also copies <z, z> to zz_keep for the next beta.
__global__ void __launch_bounds__(kCgnrThreads) k_cgnr_step(LevelArr F, MaskView m, DF y, DFc w, DF g, DFc p,
                                                            const double* __restrict__ zz,
                                                            const double* __restrict__ zp,
                                                            const double* __restrict__ ww, double* zz_keep) {
    const int ch = blockIdx.y;
    const MaskView mc = m.ch(ch);
    const double a = (ww[ch] > 0.0 && zp[ch] > 0.0) ? zp[ch] / ww[ch] : 0.0;
    float ah, al;
    df_from_d(a, ah, al);
    if (blockIdx.x == 0 && threadIdx.x == 0) zz_keep[ch] = zz[ch];
    const size_t co = (size_t)ch * F.cs;
    for (int yy = blockIdx.x; yy < F.H; yy += gridDim.x) {
        const size_t ro = co + (size_t)yy * F.pitch;
        for (int x = threadIdx.x; x < F.W; x += kCgnrThreads) {
            const size_t i = ro + x;
            float h = y.hi[i], l = y.lo[i];
            df_axpy(ah, al, w.hi[i], w.lo[i], h, l);
            y.hi[i] = h;
            y.lo[i] = l;
            if (mc.known(x, yy)) {
                float gh = g.hi[i], gl = g.lo[i];
                df_axpy(ah, al, p.hi[i], p.lo[i], gh, gl);
                g.hi[i] = gh;
                g.lo[i] = gl;
            }
        }
    }
}

// p = z + beta p on mask pixels (beta = zz / zz_old per channel, 0 on the
// first call), p = 0 elsewhere.
__global__ void __launch_bounds__(kCgnrThreads) k_cgnr_direction(LevelArr F, MaskView m, const float* __restrict__ z,
                                                                 DF p, const double* __restrict__ zz,
                                                                 const double* __restrict__ zz_old, int first) {
    const int ch = blockIdx.y;
    const MaskView mc = m.ch(ch);
    const double b = (first || !(zz_old[ch] > 0.0)) ? 0.0 : zz[ch] / zz_old[ch];
    float bh, bl;
    df_from_d(b, bh, bl);
    const size_t co = (size_t)ch * F.cs;
    for (int yy = blockIdx.x; yy < F.H; yy += gridDim.x) {
        const size_t ro = co + (size_t)yy * F.pitch;
        for (int x = threadIdx.x; x < F.W; x += kCgnrThreads) {
            const size_t i = ro + x;
            float h = 0.f, l = 0.f;
            if (mc.known(x, yy)) {
                h = z[i];
                if (!first) df_axpy(bh, bl, p.hi[i], p.lo[i], h, l);
            }
            p.hi[i] = h;
            p.lo[i] = l;
        }
    }
}

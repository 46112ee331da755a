// oras_warp.cuh -- ORAS sweep with one warp per subdomain (Sec. 3.1, Sec. 3.3).
//
// Same sweep as k_oras (oras.cuh): local operator A_i with the Robin weight
// theta at inner subdomain boundaries, local CG from v = 0 on the restricted
// residual, stop at ||r_i||^2 <= eta ||r||^2 / n_sub, restricted extension
// onto the owned core. The layout differs: a CTA is ONE warp and owns one
// 32x32 subdomain. Lane l holds the column pair c = l & 15 (columns 2c,
// 2c+1, packed in a float2) over the sixteen rows r0 .. r0+15,
// r0 = 16 (l >> 4). Vertical neighbours are register neighbours except at
// rows 15/16, which the two half-warps exchange with one xor-16 shuffle;
// horizontal neighbours outside the pair come by one shuffle per row and
// side. Every CG dot product is a warp butterfly reduction (all lanes end
// with the same value), so the loop has no shared-memory exchange and no
// barrier; shared memory holds only the 0/1 unknown-pixel mask and the
// iterate at the lane's pixels (both lane-private).
#pragma once
#include "common.cuh"
#include "oras.cuh"   // OrasArgs, shfl_xor2

constexpr int kWarpRows = 16;   // rows per lane

struct WarpGeom {
    int x0, y0, w, h;     // subdomain origin and extent (w, h <= 32)
    int c, r0;            // column pair and first row of this lane
    uint32_t um;          // bit 2k+j: pixel (row r0+k, column 2c+j) is unknown and inside
    float nwl, nwr;       // -1 where the neighbour left of 2c / right of 2c+1 is inside, else 0
    float2 dh;            // horizontal part of the diagonal for the two columns
    float dtop, dbot;     // weight of the outside neighbour above row 0 / below row h-1
    float2 dfirst, dmid, dlast;   // 32x32 subdomains: diagonal of rows k = 0, 1..14, 15
};

struct WarpShared {
    float2 msk[kWarpRows][32];     // 0/1 unknown-pixel mask per lane and row
    float2 xkeep[kWarpRows][32];   // iterate at the lane's pixels (interior subdomains)
};

// Geometry of subdomain (x0, y0) from the mask window of row `lane` held by
// each lane (all ones past the subdomain); writes the lane's mask floats.
__device__ __forceinline__ WarpGeom make_wgeom_rows(int x0, int y0, int H, int W, uint32_t wrow, float theta,
                                                    WarpShared& sh) {
    const int lane = threadIdx.x & 31;
    WarpGeom g;
    g.x0 = x0;
    g.y0 = y0;
    g.w = min(32, W - x0);
    g.h = min(32, H - y0);
    g.c = lane & 15;
    g.r0 = 16 * (lane >> 4);
    const int c0 = 2 * g.c;
    uint32_t um = 0;
#pragma unroll
    for (int k = 0; k < kWarpRows; ++k) {
        const uint32_t kn = __shfl_sync(HDI_FULL, wrow, g.r0 + k) >> c0;   // bit 0: column c0, bit 1: c0 + 1
        const bool u0 = c0 < g.w && !(kn & 1u), u1 = c0 + 1 < g.w && !(kn & 2u);
        um |= (u0 ? 1u : 0u) << (2 * k);
        um |= (u1 ? 1u : 0u) << (2 * k + 1);
        sh.msk[k][lane] = make_float2(u0 ? 1.f : 0.f, u1 ? 1.f : 0.f);
    }
    g.um = um;
    auto horiz = [&](int C) {
        const int gx = x0 + C;
        const float left = (C > 0) ? 1.f : (gx > 0 ? theta : 0.f);
        const float right = (C < g.w - 1) ? 1.f : (gx < W - 1 ? theta : 0.f);
        return left + right;
    };
    g.dh = make_float2(horiz(c0), horiz(c0 + 1));
    g.dtop = (y0 > 0) ? theta : 0.f;
    g.dbot = (y0 + g.h < H) ? theta : 0.f;
    g.nwl = (g.c > 0) ? -1.f : 0.f;
    g.nwr = (g.c < 15) ? -1.f : 0.f;
    const float vf = (g.r0 == 0) ? 1.f + g.dtop : 2.f;
    const float vl = (g.r0 + kWarpRows - 1 == 31) ? 1.f + g.dbot : 2.f;
    g.dfirst = make_float2(g.dh.x + vf, g.dh.y + vf);
    g.dmid = make_float2(g.dh.x + 2.f, g.dh.y + 2.f);
    g.dlast = make_float2(g.dh.x + vl, g.dh.y + vl);
    return g;
}

__device__ __forceinline__ WarpGeom make_wgeom(int x0, int y0, int H, int W, const MaskView& m, float theta,
                                               WarpShared& sh) {
    const int lane = threadIdx.x & 31;
    // lane l fetches the mask window of row l (rows past the subdomain read as known)
    const uint32_t wrow = (lane < min(32, H - y0)) ? m.window(x0, y0 + lane) : ~0u;
    return make_wgeom_rows(x0, y0, H, W, wrow, theta, sh);
}

template <bool FULL>
__device__ __forceinline__ float2 wdiag(const WarpGeom& g, int k) {
    if (FULL) return (k == 0) ? g.dfirst : ((k == kWarpRows - 1) ? g.dlast : g.dmid);
    const int R = g.r0 + k;
    const float v = ((R > 0) ? 1.f : g.dtop) + ((R < g.h - 1) ? 1.f : g.dbot);
    return make_float2(g.dh.x + v, g.dh.y + v);
}

// Q = A_i P on the unknown pixels (P vanishes on known and outside pixels, so
// such neighbours contribute zero). up / dn: rows r0-1 and r0+16 of P as
// this lane sees them (zero outside the subdomain).
template <bool FULL>
__device__ __forceinline__ void wapply(const WarpGeom& g, const WarpShared& sh, const float2 (&P)[kWarpRows],
                                       float2 up, float2 dn, float2 (&Q)[kWarpRows]) {
    const int lane = threadIdx.x & 31;
    const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
    for (int k = 0; k < kWarpRows; ++k) {
        const float2 mk = sh.msk[k][lane];
        const float L = __shfl_up_sync(HDI_FULL, P[k].y, 1);     // column 2c-1
        const float Rt = __shfl_down_sync(HDI_FULL, P[k].x, 1);  // column 2c+2
        float2 ns;   // minus the neighbour sum
        ns.x = fmaf(g.nwl, L, -P[k].y);
        ns.y = fmaf(g.nwr, Rt, -P[k].x);
        ns = __ffma2_rn(m1, (k > 0) ? P[k - 1] : up, ns);
        ns = __ffma2_rn(m1, (k < kWarpRows - 1) ? P[k + 1] : dn, ns);
        Q[k] = __ffma2_rn(mk, ns, __fmul2_rn(wdiag<FULL>(g, k), P[k]));
    }
}

// Sum of the lane's packed products, four accumulators (short dependency
// chains: the products of a row are ready at different times).
__device__ __forceinline__ float wdot(const float2 (&A)[kWarpRows], const float2 (&B)[kWarpRows]) {
    float2 a[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) a[j] = __fmul2_rn(A[j], B[j]);
#pragma unroll
    for (int k = 4; k < kWarpRows; ++k) a[k & 3] = __ffma2_rn(A[k], B[k], a[k & 3]);
    const float2 s01 = __fadd2_rn(a[0], a[1]), s23 = __fadd2_rn(a[2], a[3]);
    const float2 s = __fadd2_rn(s01, s23);
    return s.x + s.y;
}

// Local CG on A_i v = r from v = 0 (r: right-hand side in, final residual
// out). Stops at ||r||^2 <= thresh or after maxit iterations; returns the
// iteration count. The loop control is warp-uniform (butterfly sums).
template <bool FULL>
__device__ __forceinline__ int warp_cg(const WarpGeom& g, const WarpShared& sh, float2 (&V)[kWarpRows],
                                       float2 (&R)[kWarpRows], float thresh, int maxit) {
    const bool top = (threadIdx.x & 31) < 16;
    float2 P[kWarpRows], Q[kWarpRows];
#pragma unroll
    for (int k = 0; k < kWarpRows; ++k) {
        V[k] = make_float2(0.f, 0.f);
        P[k] = R[k];
    }
    float rr = warp_sum_f(wdot(R, R));
    const float2 z2 = make_float2(0.f, 0.f);
    int it = 0;
    while (rr > thresh && it < maxit) {
        // row 16 for the top half-warp, row 15 for the bottom one
        const float2 xo = shfl_xor2(top ? P[kWarpRows - 1] : P[0], 16);
        wapply<FULL>(g, sh, P, top ? z2 : xo, top ? xo : z2, Q);
        const float pq = warp_sum_f(wdot(P, Q));
        if (!(pq > 0.f)) break;
        const float alpha = __fdividef(rr, pq);   // CG step lengths need no IEEE rounding
        const float2 al = make_float2(alpha, alpha), nal = make_float2(-alpha, -alpha);
#pragma unroll
        for (int k = 0; k < kWarpRows; ++k) {
            V[k] = __ffma2_rn(al, P[k], V[k]);
            R[k] = __ffma2_rn(nal, Q[k], R[k]);
        }
        const float rn = warp_sum_f(wdot(R, R));
        const float beta = __fdividef(rn, rr);
        rr = rn;
        const float2 be = make_float2(beta, beta);
#pragma unroll
        for (int k = 0; k < kWarpRows; ++k) P[k] = __ffma2_rn(be, P[k], R[k]);
        ++it;
    }
    return it;
}

// One ORAS iteration (Sec. 3.1) with one warp per (subdomain, channel):
// u <- u + sum_i R~_i^T v_i, A_i v_i = R_i (b - A u); restricted extension
// onto the owned core (every output pixel written by exactly one lane).
// Arguments as k_oras; launched with 32-thread CTAs on the (nbx, nby, nch)
// grid. 12 CTAs per SM leave 168 registers per thread for the four
// 32-value vectors of the local CG.
template <bool ZERO, bool FULL>
__device__ __forceinline__ void oras_w_body(const OrasArgs& a, int bx, int by, int ch, WarpShared& sh) {
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const int x0 = sub_origin(bx, a.W, a.stride), y0 = sub_origin(by, a.H, a.stride);
    const WarpGeom g = make_wgeom(x0, y0, a.H, a.W, a.m.ch(ch), a.theta, sh);
    pdl_wait();   // x, b and the residual norm come from the preceding kernels
    const double rn2 = a.rnorm2[ch];
    const int c0 = 2 * g.c, r0 = g.r0;
    const int gx = x0 + c0;                       // absolute column of .x
    const int cx0 = min(gx, a.W - 1), cx1 = min(gx + 1, a.W - 1);
    // 8-byte aligned pair inside the image: one float2 access per row
    const bool vec = !(x0 & 1) && x0 + 32 <= a.W;
    const float* __restrict__ xin = a.xin + ch * a.cstride;
    const float* __restrict__ bb = a.b + ch * a.cstride;
    auto ld2 = [&](const float* __restrict__ p, int y) {
        const size_t row = (size_t)min(max(y, 0), a.H - 1) * a.pitch;
        if (vec) return *reinterpret_cast<const float2*>(p + row + gx);
        return make_float2(p[row + cx0], p[row + cx1]);
    };
    const bool interior = x0 > 0 && x0 + 32 < a.W && y0 > 0 && y0 + 32 < a.H;
    float2 R[kWarpRows], V[kWarpRows];
    if (interior) {
        const float* __restrict__ br = bb + (size_t)(y0 + r0) * a.pitch + gx;
        float2 B[kWarpRows];
#pragma unroll
        for (int k = 0; k < kWarpRows; ++k) B[k] = *reinterpret_cast<const float2*>(br + (size_t)k * a.pitch);
        if (ZERO) {
#pragma unroll
            for (int k = 0; k < kWarpRows; ++k) {
                R[k].x = ((g.um >> (2 * k)) & 1u) ? B[k].x : 0.f;
                R[k].y = ((g.um >> (2 * k + 1)) & 1u) ? B[k].y : 0.f;
            }
        } else {
            const float* __restrict__ xr = xin + (size_t)(y0 + r0 - 1) * a.pitch + gx;   // window row r0 - 1
            const bool hl = g.c == 0 || g.c == 15;
            const int hoff = (g.c == 0) ? -1 : 2;
            float2 X[kWarpRows + 2];
            float HV[kWarpRows];
#pragma unroll
            for (int t = 0; t < kWarpRows + 2; ++t) X[t] = *reinterpret_cast<const float2*>(xr + (size_t)t * a.pitch);
#pragma unroll
            for (int k = 0; k < kWarpRows; ++k) HV[k] = hl ? xr[(size_t)(k + 1) * a.pitch + hoff] : 0.f;
#pragma unroll
            for (int k = 0; k < kWarpRows; ++k) {
                const float2 up = X[k], xc = X[k + 1], dn = X[k + 2];
                sh.xkeep[k][lane] = xc;
                float L = __shfl_up_sync(HDI_FULL, xc.y, 1);
                float Rt = __shfl_down_sync(HDI_FULL, xc.x, 1);
                if (g.c == 0) L = HV[k];
                if (g.c == 15) Rt = HV[k];
                const float lapx = ((xc.x - L) + (xc.x - xc.y)) + ((xc.x - up.x) + (xc.x - dn.x));
                const float lapy = ((xc.y - xc.x) + (xc.y - Rt)) + ((xc.y - up.y) + (xc.y - dn.y));
                R[k].x = ((g.um >> (2 * k)) & 1u) ? (B[k].x - lapx) : 0.f;
                R[k].y = ((g.um >> (2 * k + 1)) & 1u) ? (B[k].y - lapy) : 0.f;
            }
        }
    } else {
        float2 B[kWarpRows];
#pragma unroll
        for (int k = 0; k < kWarpRows; ++k) B[k] = ld2(bb, y0 + r0 + k);
        if (ZERO) {
#pragma unroll
            for (int k = 0; k < kWarpRows; ++k) {
                R[k].x = ((g.um >> (2 * k)) & 1u) ? B[k].x : 0.f;
                R[k].y = ((g.um >> (2 * k + 1)) & 1u) ? B[k].y : 0.f;
            }
        } else {
            // R_i (b - A x) in difference form; out-of-image neighbours take
            // the centre value (zero difference). Loads first, then arithmetic.
            const bool hl = (g.c == 0 && x0 > 0) || (g.c == 15 && x0 + 32 < a.W);
            const int hcol = hl ? ((g.c == 0) ? x0 - 1 : x0 + 32) : cx0;
            float2 X[kWarpRows + 2];
            float HV[kWarpRows];
#pragma unroll
            for (int t = 0; t < kWarpRows + 2; ++t) X[t] = ld2(xin, y0 + r0 - 1 + t);
#pragma unroll
            for (int k = 0; k < kWarpRows; ++k)
                HV[k] = hl ? xin[(size_t)min(y0 + r0 + k, a.H - 1) * a.pitch + hcol] : 0.f;
            const bool in1 = gx + 1 < a.W;        // column of .y inside the image
            const bool in2 = gx + 2 < a.W;        // column right of the pair inside the image
            const bool inl = gx > 0;              // column left of the pair inside the image
#pragma unroll
            for (int k = 0; k < kWarpRows; ++k) {
                const int y = y0 + r0 + k;
                const float2 up = X[k], xc = X[k + 1], dn = X[k + 2];
                float L = __shfl_up_sync(HDI_FULL, xc.y, 1);
                float Rt = __shfl_down_sync(HDI_FULL, xc.x, 1);
                if (g.c == 0) L = hl ? HV[k] : xc.x;
                if (g.c == 15) Rt = hl ? HV[k] : xc.y;
                if (!inl) L = xc.x;
                if (!in2) Rt = xc.y;
                const float rx = in1 ? xc.y : xc.x;   // right neighbour of .x
                const bool hu = y > 0, hd = y + 1 < a.H;
                const float lapx =
                    ((xc.x - L) + (xc.x - rx)) + ((xc.x - (hu ? up.x : xc.x)) + (xc.x - (hd ? dn.x : xc.x)));
                const float lapy =
                    ((xc.y - xc.x) + (xc.y - Rt)) + ((xc.y - (hu ? up.y : xc.y)) + (xc.y - (hd ? dn.y : xc.y)));
                R[k].x = ((g.um >> (2 * k)) & 1u) ? (B[k].x - lapx) : 0.f;
                R[k].y = ((g.um >> (2 * k + 1)) & 1u) ? (B[k].y - lapy) : 0.f;
            }
        }
    }
    __syncwarp();   // the mask and the kept iterate in shared memory are read by the same lanes only
    const float thresh = (float)(rn2 * a.thresh_scale);
    const int it = warp_cg<FULL>(g, sh, V, R, thresh, a.maxit);
    if (a.iters && lane == 0 && it) atomicAdd(a.iters, (unsigned long long)it);

    if (interior) {
        // owned core [3, 29) x [3, 29) (half the overlap off every side)
        constexpr int lo = 3, hi = 29;
        const bool w0 = c0 >= lo && c0 < hi, w1 = c0 + 1 >= lo && c0 + 1 < hi;
        if (w0 || w1) {
            float* __restrict__ xo = a.xout + ch * a.cstride + (size_t)(y0 + r0) * a.pitch + gx;
#pragma unroll
            for (int k = 0; k < kWarpRows; ++k) {
                if (r0 + k >= lo && r0 + k < hi) {
                    float2 o = V[k];
                    if (!ZERO) {
                        const float2 xv = sh.xkeep[k][lane];
                        o.x += xv.x;
                        o.y += xv.y;
                    }
                    float* dst = xo + (size_t)k * a.pitch;
                    if (w0 && w1) {
                        *reinterpret_cast<float2*>(dst) = o;
                    } else {
                        if (w0) dst[0] = o.x;
                        if (w1) dst[1] = o.y;
                    }
                }
            }
        }
        return;
    }
    const int ox0 = ((bx == 0) ? 0 : bx * a.stride + a.ov / 2) - x0;
    const int ox1 = ((bx == a.nbx - 1) ? a.W : (bx + 1) * a.stride + a.ov / 2) - x0;
    const int oy0 = ((by == 0) ? 0 : by * a.stride + a.ov / 2) - y0;
    const int oy1 = ((by == a.nby - 1) ? a.H : (by + 1) * a.stride + a.ov / 2) - y0;
    const bool w0 = c0 >= ox0 && c0 < ox1, w1 = c0 + 1 >= ox0 && c0 + 1 < ox1;
    if (w0 || w1) {
        float* __restrict__ xo = a.xout + ch * a.cstride;
        if (!ZERO) {
#pragma unroll
            for (int k = 0; k < kWarpRows; ++k) {
                const float2 xv = ld2(xin, y0 + r0 + k);
                V[k].x += xv.x;
                V[k].y += xv.y;
            }
        }
#pragma unroll
        for (int k = 0; k < kWarpRows; ++k) {
            const int R0 = r0 + k;
            if (R0 >= oy0 && R0 < oy1) {
                const size_t idx = (size_t)(y0 + R0) * a.pitch + gx;
                if (w0 && w1 && vec) {
                    *reinterpret_cast<float2*>(xo + idx) = V[k];
                } else {
                    if (w0) xo[idx] = V[k].x;
                    if (w1) xo[idx + 1] = V[k].y;
                }
            }
        }
    }
}

template <bool ZERO, bool FULL>
__global__ void __launch_bounds__(32, 12) k_oras_w(OrasArgs a) {
    __shared__ WarpShared sh;
    oras_w_body<ZERO, FULL>(a, blockIdx.x, blockIdx.y, blockIdx.z, sh);
}

// One (image, channel) of a batched ORAS sweep: the sweep's arguments with
// pointers at the channel's planes (ch = 0; rnorm2[0] is the channel's
// residual norm, nbx x nby its subdomains) and whether its level is at
// least 32 x 32 (the FULL geometry).
struct OrasTask {
    OrasArgs a;
    int full;
};

// Subdomains of levels narrower or lower than 32 pixels (the coarsest levels
// of small images) take the general body through a call, so that its
// registers do not weigh on the full-size body of the batched kernel.
template <bool ZERO>
__device__ __noinline__ void oras_w_edge(const OrasArgs& a, int bx, int by, WarpShared& sh) {
    oras_w_body<ZERO, false>(a, bx, by, 0, sh);
}

// Batched ORAS sweep over tasks of different sizes, one CTA per (task,
// subdomain); the branch on the task's geometry is uniform over the CTA.
template <bool ZERO>
__global__ void __launch_bounds__(32, 12) k_oras_wb(const OrasTask* __restrict__ tasks, const int* __restrict__ cta0,
                                                  int ntasks) {
    __shared__ WarpShared sh;
    const int t = find_task(cta0, ntasks, blockIdx.x);
    const int local = blockIdx.x - cta0[t];
    const OrasArgs& a = tasks[t].a;
    const int nbx = a.nbx;
    if (tasks[t].full) oras_w_body<ZERO, true>(a, local % nbx, local / nbx, 0, sh);
    else oras_w_edge<ZERO>(a, local % nbx, local / nbx, sh);
}

// oras.cuh -- warp-per-subdomain local solves (Sec. 3.1, Sec. 3.3).
//
// One warp owns one 32x32 subdomain: lane l holds column x0+l, and each
// per-lane register array holds the 32 rows of that column. Vertical stencil
// neighbours are register neighbours, horizontal ones come from warp
// shuffles, and CG dot products are warp-shuffle reductions, so a local solve
// touches neither shared memory nor a block barrier.
//
// Local operator A_i (Sec. 3.1): the global A restricted to the subdomain,
// acting on corrections that vanish on known pixels. For an unknown pixel j
//   (A_i v)_j = d_j v_j - sum_{n in N(j) inside the subdomain} v_n,
//   d_j = #(in-image neighbours inside the subdomain)
//       + theta * #(in-image neighbours outside the subdomain).
// theta > 0 is the discrete Robin condition at inner subdomain boundaries
// (ORAS, Sec. 3.1); theta = 0 gives homogeneous Neumann conditions at every
// subdomain boundary (the local inpainting problems of RAS, Sec. 5.2).
// Out-of-image neighbours are dropped (reflecting boundary, Sec. 2.1).
#pragma once
#include "common.cuh"

struct LocalGeom {
    int x0, y0, w, h;     // subdomain origin and extent (w, h <= 32)
    uint32_t um;          // this lane's column: bit j set = row j is an unknown pixel
    float dh;             // horizontal part of d_j for this lane
    float dtop, dbot;     // weight of the outside neighbour above row 0 / below row h-1
    // full 32x32 subdomains: the diagonal of row 0, rows 1..30 and row 31,
    // with lanes 0 and 31 compensated for the shuffle returning their own value
    float d0, dmid, d31;
};

__device__ __forceinline__ float local_diag(const LocalGeom& g, int j) {
    const float up = (j > 0) ? 1.f : g.dtop;
    const float dn = (j < g.h - 1) ? 1.f : g.dbot;
    return g.dh + up + dn;
}

__device__ __forceinline__ LocalGeom make_geom(int x0, int y0, int H, int W, const MaskView& m, float theta) {
    const int lane = threadIdx.x & 31;
    LocalGeom g;
    g.x0 = x0;
    g.y0 = y0;
    g.w = min(32, W - x0);
    g.h = min(32, H - y0);
    const int gx = x0 + lane;
    const bool act = lane < g.w;
    uint32_t um = 0;
#pragma unroll 4
    for (int j = 0; j < 32; ++j) {
        if (j < g.h) {
            const uint32_t word = m.window(x0, y0 + j);
            const bool known = (word >> lane) & 1u;
            if (act && !known) um |= 1u << j;
        }
    }
    g.um = um;
    const float left = (lane > 0) ? 1.f : (gx > 0 ? theta : 0.f);
    const float right = (lane < g.w - 1) ? 1.f : (gx < W - 1 ? theta : 0.f);
    g.dh = left + right;
    g.dtop = (y0 > 0) ? theta : 0.f;
    g.dbot = (y0 + g.h < H) ? theta : 0.f;
    const float dhc = g.dh + ((lane == 0) ? 1.f : 0.f) + ((lane == 31) ? 1.f : 0.f);
    g.d0 = dhc + 1.f + g.dtop;
    g.dmid = dhc + 2.f;
    g.d31 = dhc + 1.f + g.dbot;
    return g;
}

// q = A_i p on the unknown pixels (p is zero on known / invalid pixels).
// FULL: the subdomain is 32x32, so the row diagonal is known at compile time
// and the edge lanes keep the value the shuffle returns (their own p, which
// d0/dmid/d31 compensate) instead of selecting zero.
template <bool FULL>
__device__ __forceinline__ void local_apply(const LocalGeom& g, const float (&p)[32], float (&q)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        float pl = __shfl_up_sync(HDI_FULL, p[j], 1);
        float pr = __shfl_down_sync(HDI_FULL, p[j], 1);
        if (!FULL) {
            if (lane == 0) pl = 0.f;
            if (lane == 31) pr = 0.f;
        }
        float s = pl + pr;
        if (j > 0) s += p[j - 1];
        if (j < 31) s += p[j + 1];
        float d;
        if (FULL) d = (j == 0) ? g.d0 : ((j == 31) ? g.d31 : g.dmid);
        else d = local_diag(g, j);
        const float v = d * p[j] - s;
        q[j] = ((g.um >> j) & 1u) ? v : 0.f;
    }
}

// Conjugate gradients on A_i v = r (v starts at 0; r holds the right-hand
// side on entry and the final residual on exit). Stops when ||r||^2 <= thresh
// or after maxit iterations; returns the iteration count.
template <bool FULL>
__device__ __forceinline__ int local_cg(const LocalGeom& g, float (&v)[32], float (&r)[32], float thresh, int maxit) {
    float p[32], q[32];
    float rr = 0.f;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        v[j] = 0.f;
        p[j] = r[j];
        rr += r[j] * r[j];
    }
    rr = warp_sum_f(rr);
    int it = 0;
    while (rr > thresh && it < maxit) {
        local_apply<FULL>(g, p, q);
        float pq = 0.f;
#pragma unroll
        for (int j = 0; j < 32; ++j) pq += p[j] * q[j];
        pq = warp_sum_f(pq);
        if (!(pq > 0.f)) break;
        const float alpha = rr / pq;
        float rn = 0.f;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            v[j] += alpha * p[j];
            r[j] -= alpha * q[j];
            rn += r[j] * r[j];
        }
        rn = warp_sum_f(rn);
        const float beta = rn / rr;
        rr = rn;
#pragma unroll
        for (int j = 0; j < 32; ++j) p[j] = r[j] + beta * p[j];
        ++it;
    }
    return it;
}

struct OrasArgs {
    MaskView m;
    int H, W, pitch;           // level size, floats per row
    long long cstride;         // floats per channel
    int nch;
    int nbx, nby, stride, ov;
    float theta;
    int maxit;
    double thresh_scale;       // eta / (subdomains per channel)
    const float* xin;          // iterate before the sweep (ignored when ZERO)
    float* xout;               // iterate after the sweep (never aliases xin)
    const float* b;            // right-hand side on this level
    const double* rnorm2;      // [nch] global ||b - A xin||^2
    unsigned long long* iters; // optional: total local CG iterations
};

// Launch bounds: 4 CTAs per SM caps the register file at 128 per thread
// (16 warps per SM; the compiler spills a few values of the local CG to L1),
// which measured faster than 255 registers at 8 warps per SM.
// One ORAS iteration (Sec. 3.1): u <- u + sum_i R~_i^T v_i with
// A_i v_i = R_i (b - A u). Restricted extension: each pixel takes the
// correction of the one subdomain whose core (the subdomain minus half the
// overlap on each inner side) contains it, so every output pixel is written
// by exactly one warp and the sweep needs no atomics.
template <bool ZERO, bool FULL>
__global__ void __launch_bounds__(128, 4) k_oras(OrasArgs a) {
    const int wid = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int nb = a.nbx * a.nby;
    if (wid >= nb * a.nch) return;
    const int ch = wid / nb;
    const int bi = wid - ch * nb;
    const int by = bi / a.nbx;
    const int bx = bi - by * a.nbx;
    const int x0 = sub_origin(bx, a.W, a.stride), y0 = sub_origin(by, a.H, a.stride);
    const LocalGeom g = make_geom(x0, y0, a.H, a.W, a.m.ch(ch), a.theta);
    const int gx = x0 + lane;
    const bool act = lane < g.w;
    const int gxc = act ? gx : (a.W - 1);   // clamped column for safe loads
    const float* xin = a.xin + ch * a.cstride;
    const float* bb = a.b + ch * a.cstride;

    float r[32], v[32];
    if (ZERO) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int y = min(y0 + j, a.H - 1);
            const float bv = bb[(size_t)y * a.pitch + gxc];
            r[j] = ((g.um >> j) & 1u) ? bv : 0.f;
        }
    } else {
        // R_i (b - A x) in difference form (sum of neighbour differences).
        const bool has_l = (lane == 0) && (gx > 0);
        const bool has_r = (lane == g.w - 1) && (gx + 1 < a.W);
        float xu = xin[(size_t)max(y0 - 1, 0) * a.pitch + gxc];
        float xc = xin[(size_t)y0 * a.pitch + gxc];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int y = min(y0 + j, a.H - 1);
            const int yn = min(y + 1, a.H - 1);
            const float xd = xin[(size_t)yn * a.pitch + gxc];
            float xl = __shfl_up_sync(HDI_FULL, xc, 1);
            float xr = __shfl_down_sync(HDI_FULL, xc, 1);
            if (lane == 0) xl = has_l ? xin[(size_t)y * a.pitch + gx - 1] : xc;
            if (has_r) xr = xin[(size_t)y * a.pitch + gx + 1];
            else if (lane == g.w - 1) xr = xc;
            const float bv = bb[(size_t)y * a.pitch + gxc];
            const float up = (y > 0) ? xu : xc;
            const float dn = (y + 1 < a.H) ? xd : xc;
            const float lap = ((xc - xl) + (xc - xr)) + ((xc - up) + (xc - dn));
            r[j] = ((g.um >> j) & 1u) ? (bv - lap) : 0.f;
            xu = xc;
            xc = xd;
        }
    }
    const float thresh = (float)(a.rnorm2[ch] * a.thresh_scale);
    const int it = local_cg<FULL>(g, v, r, thresh, a.maxit);
    if (a.iters && lane == 0 && it) atomicAdd(a.iters, (unsigned long long)it);

    // owned core in absolute coordinates, then relative to the (possibly
    // shifted) origin
    const int ox0 = ((bx == 0) ? 0 : bx * a.stride + a.ov / 2) - x0;
    const int ox1 = ((bx == a.nbx - 1) ? a.W : (bx + 1) * a.stride + a.ov / 2) - x0;
    const int oy0 = ((by == 0) ? 0 : by * a.stride + a.ov / 2) - y0;
    const int oy1 = ((by == a.nby - 1) ? a.H : (by + 1) * a.stride + a.ov / 2) - y0;
    if (lane >= ox0 && lane < ox1) {
        float* xo = a.xout + ch * a.cstride;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (j >= oy0 && j < oy1) {
                const size_t idx = (size_t)(y0 + j) * a.pitch + gx;
                xo[idx] = ZERO ? v[j] : (xin[idx] + v[j]);
            }
        }
    }
}

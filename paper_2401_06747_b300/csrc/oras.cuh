// oras.cuh -- warp-per-subdomain local solves (Sec. 3.1, Sec. 3.3).
//
// One warp owns one 32x32 subdomain. Lane l holds the column pair
// c = l & 15 (columns 2c and 2c+1) over the row half hh = l >> 4 (rows
// 16hh .. 16hh+15); every per-lane array holds 16 float2 values, column 2c
// in .x and 2c+1 in .y. The pair layout puts two pixels of one row in a
// 64-bit register pair, so the vector updates and most of the stencil run as
// packed FP32x2 operations (two results per instruction), and a lane needs
// one shuffle per row and side for its horizontal neighbours (the inner
// neighbours of the pair are its own registers). Vertical neighbours are
// register neighbours, except across the two row halves (one xor-16 shuffle
// per apply), and CG dot products are warp-shuffle reductions: a local solve
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
    int c, hh;            // this lane's column pair and row half
    uint32_t um;          // bit 2k+j: pixel (row 16hh+k, column 2c+j) is unknown and inside
    // -1 where the neighbour lies in the subdomain, else 0: left of column
    // 2c, right of column 2c+1, above row 0 / below row 15 of this half
    float nwl, nwr, nwu, nwd;
    float2 dh;            // horizontal part of d_j for the two columns
    float dtop, dbot;     // weight of the outside neighbour above row 0 / below row h-1
    float2 dfirst, dmid, dlast;   // 32x32 subdomains: diagonal of rows k = 0, 1..14, 15
};

// Per-warp shared-memory slab of the local CG: the 0/1 unknown-pixel mask of
// the lane's 32 pixels as float2 (lane-private: each lane reads back only
// what it wrote, so no synchronisation is needed). Multiplying by it inside
// the packed stencil replaces a per-pixel bit test and select.
constexpr int kLocalSlab = 16 * 32;   // float2 per warp

// Geometry of subdomain (x0, y0); writes the lane's mask floats to msk[k * 32]
// (msk = warp slab + lane).
__device__ __forceinline__ LocalGeom make_geom(int x0, int y0, int H, int W, const MaskView& m, float theta,
                                               float2* msk) {
    const int lane = threadIdx.x & 31;
    LocalGeom g;
    g.x0 = x0;
    g.y0 = y0;
    g.w = min(32, W - x0);
    g.h = min(32, H - y0);
    g.c = lane & 15;
    g.hh = lane >> 4;
    const int c0 = 2 * g.c, r0 = 16 * g.hh;
    // lane l fetches the mask word of row l (rows past the subdomain read as known)
    const uint32_t wrow = (lane < g.h) ? m.window(x0, y0 + lane) : ~0u;
    uint32_t um = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const uint32_t kn = __shfl_sync(HDI_FULL, wrow, r0 + k) >> c0;   // bit 0: column c0, bit 1: c0 + 1
        const bool u0 = c0 < g.w && !(kn & 1u), u1 = c0 + 1 < g.w && !(kn & 2u);
        um |= (u0 ? 1u : 0u) << (2 * k);
        um |= (u1 ? 1u : 0u) << (2 * k + 1);
        msk[k * 32] = make_float2(u0 ? 1.f : 0.f, u1 ? 1.f : 0.f);
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
    g.nwu = g.hh ? -1.f : 0.f;
    g.nwd = g.hh ? 0.f : -1.f;
    const float vf = g.hh ? 2.f : 1.f + g.dtop;
    const float vl = g.hh ? 1.f + g.dbot : 2.f;
    g.dfirst = make_float2(g.dh.x + vf, g.dh.y + vf);
    g.dmid = make_float2(g.dh.x + 2.f, g.dh.y + 2.f);
    g.dlast = make_float2(g.dh.x + vl, g.dh.y + vl);
    return g;
}

// Diagonal of row k of this lane's half (both columns).
template <bool FULL>
__device__ __forceinline__ float2 local_diag(const LocalGeom& g, int k) {
    if (FULL) return (k == 0) ? g.dfirst : ((k == 15) ? g.dlast : g.dmid);
    const int R = 16 * g.hh + k;
    const float v = ((R > 0) ? 1.f : g.dtop) + ((R < g.h - 1) ? 1.f : g.dbot);
    return make_float2(g.dh.x + v, g.dh.y + v);
}

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
    return make_float2(__shfl_xor_sync(HDI_FULL, v.x, m), __shfl_xor_sync(HDI_FULL, v.y, m));
}

// Q = A_i P on the unknown pixels (P is zero on known / outside pixels, so
// shuffles that fetch such pixels contribute zero; neighbours outside the
// subdomain carry weight 0). Q = d P + M (-neighbour sum) with M the 0/1
// mask: on a known pixel P = 0 and M = 0, so Q = 0 there.
template <bool FULL>
__device__ __forceinline__ void local_apply(const LocalGeom& g, const float2* __restrict__ msk,
                                            const float2 (&P)[16], float2 (&Q)[16]) {
    const float2 U = shfl_xor2(P[15], 16);   // row 15 of the upper half (used by the lower half)
    const float2 D = shfl_xor2(P[0], 16);    // row 16 of the lower half (used by the upper half)
    const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const float2 mk = msk[k * 32];
        const float L = __shfl_up_sync(HDI_FULL, P[k].y, 1);     // column 2c-1
        const float Rt = __shfl_down_sync(HDI_FULL, P[k].x, 1);  // column 2c+2
        float2 ns;   // minus the neighbour sum
        ns.x = fmaf(g.nwl, L, -P[k].y);
        ns.y = fmaf(g.nwr, Rt, -P[k].x);
        if (k > 0) ns = __ffma2_rn(m1, P[k - 1], ns);
        else ns = __ffma2_rn(make_float2(g.nwu, g.nwu), U, ns);
        if (k < 15) ns = __ffma2_rn(m1, P[k + 1], ns);
        else ns = __ffma2_rn(make_float2(g.nwd, g.nwd), D, ns);
        Q[k] = __ffma2_rn(mk, ns, __fmul2_rn(local_diag<FULL>(g, k), P[k]));
    }
}

// Conjugate gradients on A_i v = r (v starts at 0; r holds the right-hand
// side on entry and the final residual on exit). Stops when ||r||^2 <= thresh
// or after maxit iterations; returns the iteration count.
template <bool FULL>
__device__ __forceinline__ int local_cg(const LocalGeom& g, const float2* __restrict__ msk, float2 (&V)[16],
                                        float2 (&R)[16], float thresh, int maxit) {
    float2 P[16], Q[16];
    float2 a0 = make_float2(0.f, 0.f), a1 = a0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        V[k] = make_float2(0.f, 0.f);
        P[k] = R[k];
        if (k & 1) a1 = __ffma2_rn(R[k], R[k], a1);
        else a0 = __ffma2_rn(R[k], R[k], a0);
    }
    float rr = warp_sum_f((a0.x + a0.y) + (a1.x + a1.y));
    int it = 0;
    while (rr > thresh && it < maxit) {
        local_apply<FULL>(g, msk, P, Q);
        a0 = make_float2(0.f, 0.f);
        a1 = a0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (k & 1) a1 = __ffma2_rn(P[k], Q[k], a1);
            else a0 = __ffma2_rn(P[k], Q[k], a0);
        }
        const float pq = warp_sum_f((a0.x + a0.y) + (a1.x + a1.y));
        if (!(pq > 0.f)) break;
        const float alpha = rr / pq;
        const float2 al = make_float2(alpha, alpha), nal = make_float2(-alpha, -alpha);
        a0 = make_float2(0.f, 0.f);
        a1 = a0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            V[k] = __ffma2_rn(al, P[k], V[k]);
            R[k] = __ffma2_rn(nal, Q[k], R[k]);
            if (k & 1) a1 = __ffma2_rn(R[k], R[k], a1);
            else a0 = __ffma2_rn(R[k], R[k], a0);
        }
        const float rn = warp_sum_f((a0.x + a0.y) + (a1.x + a1.y));
        const float beta = rn / rr;
        rr = rn;
        const float2 be = make_float2(beta, beta);
#pragma unroll
        for (int k = 0; k < 16; ++k) P[k] = __ffma2_rn(be, P[k], R[k]);
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

// Launch bounds: 3 CTAs of 4 warps per SM leave 168 registers per thread,
// enough for the four 32-value vectors of the local CG without spills.
// One ORAS iteration (Sec. 3.1): u <- u + sum_i R~_i^T v_i with
// A_i v_i = R_i (b - A u). Restricted extension: each pixel takes the
// correction of the one subdomain whose core (the subdomain minus half the
// overlap on each inner side) contains it, so every output pixel is written
// by exactly one warp and the sweep needs no atomics.
template <bool ZERO, bool FULL>
__global__ void __launch_bounds__(128, 3) k_oras(OrasArgs a) {
    __shared__ float2 slab[4 * kLocalSlab];
    const int wid = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int nb = a.nbx * a.nby;
    if (wid >= nb * a.nch) return;
    const int ch = wid / nb;
    const int bi = wid - ch * nb;
    const int by = bi / a.nbx;
    const int bx = bi - by * a.nbx;
    const int x0 = sub_origin(bx, a.W, a.stride), y0 = sub_origin(by, a.H, a.stride);
    const double rn2 = a.rnorm2[ch];
    float2* msk = slab + (threadIdx.x >> 5) * kLocalSlab + (threadIdx.x & 31);
    const LocalGeom g = make_geom(x0, y0, a.H, a.W, a.m.ch(ch), a.theta, msk);
    const int c0 = 2 * g.c, r0 = 16 * g.hh;
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

    float2 R[16], V[16];
    {
        float2 B[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) B[k] = ld2(bb, y0 + r0 + k);
        if (ZERO) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                R[k].x = ((g.um >> (2 * k)) & 1u) ? B[k].x : 0.f;
                R[k].y = ((g.um >> (2 * k + 1)) & 1u) ? B[k].y : 0.f;
            }
        } else {
            // R_i (b - A x) in difference form (sum of neighbour differences);
            // out-of-image neighbours take the centre value (zero difference).
            // All loads are issued before the arithmetic.
            const bool hl = (g.c == 0 && x0 > 0) || (g.c == 15 && x0 + 32 < a.W);
            const int hcol = hl ? ((g.c == 0) ? x0 - 1 : x0 + 32) : cx0;
            float2 X[18];
            float HV[16];
#pragma unroll
            for (int t = 0; t < 18; ++t) X[t] = ld2(xin, y0 + r0 - 1 + t);
#pragma unroll
            for (int k = 0; k < 16; ++k)
                HV[k] = hl ? xin[(size_t)min(y0 + r0 + k, a.H - 1) * a.pitch + hcol] : 0.f;
            const bool in1 = gx + 1 < a.W;        // column of .y inside the image
            const bool in2 = gx + 2 < a.W;        // column right of the pair inside the image
            const bool inl = gx > 0;              // column left of the pair inside the image
#pragma unroll
            for (int k = 0; k < 16; ++k) {
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
    const float thresh = (float)(rn2 * a.thresh_scale);
    const int it = local_cg<FULL>(g, msk, V, R, thresh, a.maxit);
    if (a.iters && (threadIdx.x & 31) == 0 && it) atomicAdd(a.iters, (unsigned long long)it);

    // owned core in absolute coordinates, then relative to the (possibly
    // shifted) origin
    const int ox0 = ((bx == 0) ? 0 : bx * a.stride + a.ov / 2) - x0;
    const int ox1 = ((bx == a.nbx - 1) ? a.W : (bx + 1) * a.stride + a.ov / 2) - x0;
    const int oy0 = ((by == 0) ? 0 : by * a.stride + a.ov / 2) - y0;
    const int oy1 = ((by == a.nby - 1) ? a.H : (by + 1) * a.stride + a.ov / 2) - y0;
    const bool w0 = c0 >= ox0 && c0 < ox1, w1 = c0 + 1 >= ox0 && c0 + 1 < ox1;
    if (w0 || w1) {
        float* __restrict__ xo = a.xout + ch * a.cstride;
        if (!ZERO) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const float2 xv = ld2(xin, y0 + r0 + k);
                V[k].x += xv.x;
                V[k].y += xv.y;
            }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
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

// oras.cuh -- subdomain local solves (Sec. 3.1, Sec. 3.3).
//
// One CTA of two warps owns one 32x32 subdomain. Thread t = 32 w + l holds
// the column pair c = l & 15 (columns 2c, 2c+1) over the eight rows
// r0 .. r0+7, r0 = 16 w + 8 (l >> 4): per-thread arrays hold 8 float2
// values, column 2c in .x and 2c+1 in .y. The pair layout puts two pixels of
// a row in a 64-bit register pair, so the vector updates and most of the
// stencil run as packed FP32x2 operations; horizontal neighbours outside the
// pair come by one shuffle per row and side, vertical ones are register
// neighbours, the row octets of a warp meet by an xor-16 shuffle, and the two
// warps meet at rows 15/16 through shared memory. CG dot products are warp
// reductions plus one shared-memory exchange, and each iteration has two CTA
// barriers: the boundary rows for the next stencil travel with the second
// reduction (the neighbour warp's residual and old search direction, from
// which each thread forms the new direction itself).
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

constexpr int kLocalThreads = 64;   // threads per subdomain (two warps)

struct LocalGeom {
    int x0, y0, w, h;     // subdomain origin and extent (w, h <= 32)
    int c, r0;            // this thread's column pair and first row
    uint32_t um;          // bit 2k+j: pixel (row r0+k, column 2c+j) is unknown and inside
    // -1 where the neighbour lies in the subdomain, else 0: left of column
    // 2c, right of column 2c+1, above row r0 / below row r0+7
    float nwl, nwr, nwu, nwd;
    float2 dh;            // horizontal part of d_j for the two columns
    float dtop, dbot;     // weight of the outside neighbour above row 0 / below row h-1
    float2 dfirst, dmid, dlast;   // 32x32 subdomains: diagonal of rows k = 0, 1..6, 7
};

// Shared memory of one subdomain's local CG.
struct LocalShared {
    float2 msk[8][kLocalThreads];  // 0/1 unknown-pixel mask per thread and row (thread-private)
    float2 seam[2][2][2][16];      // [parity][side: 0 = row 15, 1 = row 16][R, P_old][column pair]
    float red[5][2];               // warp partial sums: pq / rn by parity, initial rr
    float2 xkeep[8][kLocalThreads]; // iterate at the thread's pixels (interior sweeps: reused by the output)
};

// Geometry of subdomain (x0, y0); writes the thread's mask floats.
__device__ __forceinline__ LocalGeom make_geom(int x0, int y0, int H, int W, const MaskView& m, float theta,
                                               LocalShared& sh) {
    const int t = threadIdx.x;
    const int lane = t & 31;
    LocalGeom g;
    g.x0 = x0;
    g.y0 = y0;
    g.w = min(32, W - x0);
    g.h = min(32, H - y0);
    g.c = lane & 15;
    g.r0 = 16 * (t >> 5) + 8 * (lane >> 4);
    const int c0 = 2 * g.c;
    // lane l < 16 of warp w fetches the mask word of row 16 w + l, the warp's
    // rows (rows past the subdomain read as known)
    const int wr = 16 * (t >> 5) + (lane & 15);
    const uint32_t wrow = (lane < 16 && wr < g.h) ? m.window(x0, y0 + wr) : ~0u;
    uint32_t um = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t kn = __shfl_sync(HDI_FULL, wrow, g.r0 - 16 * (t >> 5) + k) >> c0;   // bit 0: column c0, bit 1: c0 + 1
        const bool u0 = c0 < g.w && !(kn & 1u), u1 = c0 + 1 < g.w && !(kn & 2u);
        um |= (u0 ? 1u : 0u) << (2 * k);
        um |= (u1 ? 1u : 0u) << (2 * k + 1);
        sh.msk[k][t] = make_float2(u0 ? 1.f : 0.f, u1 ? 1.f : 0.f);
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
    g.nwu = (g.r0 > 0) ? -1.f : 0.f;
    g.nwd = (g.r0 + 8 < 32) ? -1.f : 0.f;
    const float vf = (g.r0 == 0) ? 1.f + g.dtop : 2.f;
    const float vl = (g.r0 + 7 == 31) ? 1.f + g.dbot : 2.f;
    g.dfirst = make_float2(g.dh.x + vf, g.dh.y + vf);
    g.dmid = make_float2(g.dh.x + 2.f, g.dh.y + 2.f);
    g.dlast = make_float2(g.dh.x + vl, g.dh.y + vl);
    return g;
}

// Diagonal of row r0 + k (both columns).
template <bool FULL>
__device__ __forceinline__ float2 local_diag(const LocalGeom& g, int k) {
    if (FULL) return (k == 0) ? g.dfirst : ((k == 7) ? g.dlast : g.dmid);
    const int R = g.r0 + k;
    const float v = ((R > 0) ? 1.f : g.dtop) + ((R < g.h - 1) ? 1.f : g.dbot);
    return make_float2(g.dh.x + v, g.dh.y + v);
}

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
    return make_float2(__shfl_xor_sync(HDI_FULL, v.x, m), __shfl_xor_sync(HDI_FULL, v.y, m));
}

// Sum over the CTA of one value per thread: warp sums, exchanged through
// red[slot] across one barrier, added in a fixed order (every thread gets the
// same result).
__device__ __forceinline__ float cta_sum2(float v, LocalShared& sh, int slot) {
    v = warp_sum_f(v);
    if ((threadIdx.x & 31) == 0) sh.red[slot][threadIdx.x >> 5] = v;
    __syncthreads();
    return sh.red[slot][0] + sh.red[slot][1];
}

// Q = A_i P on the unknown pixels (P is zero on known / outside pixels, so
// fetched neighbours of that kind contribute zero; neighbours outside the
// subdomain carry weight 0). Q = d P + M (-neighbour sum) with M the 0/1
// mask: on a known pixel P = 0 and M = 0, so Q = 0 there. Nb = rows r0-1
// and r0+8 of P as seen by this thread (from the other octet or warp).
template <bool FULL>
__device__ __forceinline__ void local_apply(const LocalGeom& g, const LocalShared& sh, const float2 (&P)[8],
                                            float2 up, float2 dn, float2 (&Q)[8]) {
    const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float2 mk = sh.msk[k][threadIdx.x];
        const float L = __shfl_up_sync(HDI_FULL, P[k].y, 1);     // column 2c-1
        const float Rt = __shfl_down_sync(HDI_FULL, P[k].x, 1);  // column 2c+2
        float2 ns;   // minus the neighbour sum
        ns.x = fmaf(g.nwl, L, -P[k].y);
        ns.y = fmaf(g.nwr, Rt, -P[k].x);
        if (k > 0) ns = __ffma2_rn(m1, P[k - 1], ns);
        else ns = __ffma2_rn(make_float2(g.nwu, g.nwu), up, ns);
        if (k < 7) ns = __ffma2_rn(m1, P[k + 1], ns);
        else ns = __ffma2_rn(make_float2(g.nwd, g.nwd), dn, ns);
        Q[k] = __ffma2_rn(mk, ns, __fmul2_rn(local_diag<FULL>(g, k), P[k]));
    }
}

// Conjugate gradients on A_i v = r (v starts at 0; r holds the right-hand
// side on entry and the final residual on exit). Stops when ||r||^2 <= thresh
// or after maxit iterations; returns the iteration count. Called by all 64
// threads of the CTA (the loop control is uniform: every thread holds the
// same reduced values).
template <bool FULL>
__device__ __forceinline__ int local_cg(const LocalGeom& g, LocalShared& sh, float2 (&V)[8], float2 (&R)[8],
                                        float thresh, int maxit) {
    const int t = threadIdx.x, lane = t & 31, wv = t >> 5, oct = lane >> 4;
    // boundary rows exchanged between the warps: octet 1 of warp 0 owns
    // row 15 (k = 7), octet 0 of warp 1 owns row 16 (k = 0)
    const bool w15 = (wv == 0 && oct == 1), w16 = (wv == 1 && oct == 0);
    float2 P[8], Q[8];
    float2 a0 = make_float2(0.f, 0.f), a1 = a0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        V[k] = make_float2(0.f, 0.f);
        P[k] = R[k];
        if (k & 1) a1 = __ffma2_rn(R[k], R[k], a1);
        else a0 = __ffma2_rn(R[k], R[k], a0);
    }
    const float2 z2 = make_float2(0.f, 0.f);
    if (w15) { sh.seam[0][0][0][g.c] = R[7]; sh.seam[0][0][1][g.c] = z2; }
    if (w16) { sh.seam[0][1][0][g.c] = R[0]; sh.seam[0][1][1][g.c] = z2; }
    float rr = cta_sum2((a0.x + a0.y) + (a1.x + a1.y), sh, 4);
    float beta = 0.f;   // P = R + beta * P_old for the rows in the seam buffer
    int it = 0;
    while (rr > thresh && it < maxit) {
        const int par = it & 1;
        // rows r0-1 / r0+8: one comes from the other octet of the warp (octet
        // 0 sends its last row, octet 1 its first, one exchange), the other
        // from the other warp through shared memory (octet 0 takes row 15,
        // octet 1 row 16: one pair of loads, addressed by the octet)
        const float2 xo = shfl_xor2((oct == 0) ? P[7] : P[0], 16);
        const float2 b2 = make_float2(beta, beta);
        const float2 sn = __ffma2_rn(b2, sh.seam[par][oct][1][g.c], sh.seam[par][oct][0][g.c]);
        const float2 up = (oct == 0) ? sn : xo, dn = (oct == 1) ? sn : xo;
        local_apply<FULL>(g, sh, P, up, dn, Q);
        a0 = make_float2(0.f, 0.f);
        a1 = a0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (k & 1) a1 = __ffma2_rn(P[k], Q[k], a1);
            else a0 = __ffma2_rn(P[k], Q[k], a0);
        }
        const float pq = cta_sum2((a0.x + a0.y) + (a1.x + a1.y), sh, par * 2);
        if (!(pq > 0.f)) break;
        const float alpha = __fdividef(rr, pq);   // CG step lengths need no IEEE rounding
        const float2 al = make_float2(alpha, alpha), nal = make_float2(-alpha, -alpha);
        a0 = make_float2(0.f, 0.f);
        a1 = a0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            V[k] = __ffma2_rn(al, P[k], V[k]);
            R[k] = __ffma2_rn(nal, Q[k], R[k]);
            if (k & 1) a1 = __ffma2_rn(R[k], R[k], a1);
            else a0 = __ffma2_rn(R[k], R[k], a0);
        }
        const int npar = par ^ 1;
        if (w15) { sh.seam[npar][0][0][g.c] = R[7]; sh.seam[npar][0][1][g.c] = P[7]; }
        if (w16) { sh.seam[npar][1][0][g.c] = R[0]; sh.seam[npar][1][1][g.c] = P[0]; }
        const float rn = cta_sum2((a0.x + a0.y) + (a1.x + a1.y), sh, par * 2 + 1);
        beta = __fdividef(rn, rr);
        rr = rn;
        const float2 be = make_float2(beta, beta);
#pragma unroll
        for (int k = 0; k < 8; ++k) P[k] = __ffma2_rn(be, P[k], R[k]);
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

// One ORAS iteration (Sec. 3.1): u <- u + sum_i R~_i^T v_i with
// A_i v_i = R_i (b - A u). Restricted extension: each pixel takes the
// correction of the one subdomain whose core (the subdomain minus half the
// overlap on each inner side) contains it, so every output pixel is written
// by exactly one thread and the sweep needs no atomics.
// One CTA per (subdomain, channel); 10 CTAs per SM leave 102 registers per
// thread, enough for the four 16-value vectors of the local CG.
template <bool ZERO, bool FULL>
__global__ void __launch_bounds__(kLocalThreads, 10) k_oras(OrasArgs a) {
    __shared__ LocalShared sh;
    pdl_trigger();
    const int bx = blockIdx.x, by = blockIdx.y, ch = blockIdx.z;   // grid (nbx, nby, nch)
    const int x0 = sub_origin(bx, a.W, a.stride), y0 = sub_origin(by, a.H, a.stride);
    const LocalGeom g = make_geom(x0, y0, a.H, a.W, a.m.ch(ch), a.theta, sh);
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

    // Interior subdomains (all neighbours and the halo inside the image; x0 is
    // then a multiple of the stride, so even) take a path without clamping or
    // boundary selects; the others the general one.
    const bool interior = x0 > 0 && x0 + 32 < a.W && y0 > 0 && y0 + 32 < a.H;
    float2 R[8], V[8];
    if (interior) {
        const float* __restrict__ xr = xin + (size_t)(y0 + r0 - 1) * a.pitch + gx;   // window row r0 - 1
        const float* __restrict__ br = bb + (size_t)(y0 + r0) * a.pitch + gx;
        float2 B[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) B[k] = *reinterpret_cast<const float2*>(br + (size_t)k * a.pitch);
        if (ZERO) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                R[k].x = ((g.um >> (2 * k)) & 1u) ? B[k].x : 0.f;
                R[k].y = ((g.um >> (2 * k + 1)) & 1u) ? B[k].y : 0.f;
            }
        } else {
            const bool hl = g.c == 0 || g.c == 15;
            const int hoff = (g.c == 0) ? -1 : 2;
            float2 X[10];
            float HV[8];
#pragma unroll
            for (int t = 0; t < 10; ++t) X[t] = *reinterpret_cast<const float2*>(xr + (size_t)t * a.pitch);
#pragma unroll
            for (int k = 0; k < 8; ++k) HV[k] = hl ? xr[(size_t)(k + 1) * a.pitch + hoff] : 0.f;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float2 up = X[k], xc = X[k + 1], dn = X[k + 2];
                sh.xkeep[k][threadIdx.x] = xc;
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
        float2 B[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) B[k] = ld2(bb, y0 + r0 + k);
        if (ZERO) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                R[k].x = ((g.um >> (2 * k)) & 1u) ? B[k].x : 0.f;
                R[k].y = ((g.um >> (2 * k + 1)) & 1u) ? B[k].y : 0.f;
            }
        } else {
            // R_i (b - A x) in difference form (sum of neighbour differences);
            // out-of-image neighbours take the centre value (zero difference).
            // All loads are issued before the arithmetic.
            const bool hl = (g.c == 0 && x0 > 0) || (g.c == 15 && x0 + 32 < a.W);
            const int hcol = hl ? ((g.c == 0) ? x0 - 1 : x0 + 32) : cx0;
            float2 X[10];
            float HV[8];
#pragma unroll
            for (int t = 0; t < 10; ++t) X[t] = ld2(xin, y0 + r0 - 1 + t);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                HV[k] = hl ? xin[(size_t)min(y0 + r0 + k, a.H - 1) * a.pitch + hcol] : 0.f;
            const bool in1 = gx + 1 < a.W;        // column of .y inside the image
            const bool in2 = gx + 2 < a.W;        // column right of the pair inside the image
            const bool inl = gx > 0;              // column left of the pair inside the image
#pragma unroll
            for (int k = 0; k < 8; ++k) {
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
    const int it = local_cg<FULL>(g, sh, V, R, thresh, a.maxit);
    if (a.iters && threadIdx.x == 0 && it) atomicAdd(a.iters, (unsigned long long)it);

    if (interior) {
        // owned core [3, 29) x [3, 29) (half the overlap off every side)
        constexpr int lo = 3, hi = 29;
        const bool w0 = c0 >= lo && c0 < hi, w1 = c0 + 1 >= lo && c0 + 1 < hi;
        if (w0 || w1) {
            float* __restrict__ xo = a.xout + ch * a.cstride + (size_t)(y0 + r0) * a.pitch + gx;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (r0 + k >= lo && r0 + k < hi) {
                    float2 o = V[k];
                    if (!ZERO) {
                        const float2 xv = sh.xkeep[k][threadIdx.x];
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
            for (int k = 0; k < 8; ++k) {
                const float2 xv = ld2(xin, y0 + r0 + k);
                V[k].x += xv.x;
                V[k].y += xv.y;
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
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

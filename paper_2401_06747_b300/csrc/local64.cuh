// local64.cuh -- local inpainting echoes on 64x64 subdomains (the RAS block
// size of Sec. 5.2: 64 with overlap 6), for tonal optimisation at sparse
// masks, where the 32x32 blocks couple too weakly.
//
// One CTA of eight warps owns a 64x64 subdomain. Lane l of warp w holds the
// column pair (2l, 2l+1) over the eight rows 8w .. 8w+7 (per-thread arrays of
// 8 float2, as in the 32x32 layout); horizontal neighbours outside the pair
// come by shuffles across the warp, vertical ones are register neighbours
// inside a warp and shared-memory boundary rows between warps. The local
// operator is the Neumann one of Sec. 5.2 (theta = 0): for an unknown pixel j
// of the subdomain, (A_i v)_j = d_j v_j - sum of v over its unknown
// neighbours inside the subdomain, d_j = number of its neighbours inside the
// subdomain (known ones included, their v being 0). CG with two barriers per
// iteration; each warp's boundary rows travel with the second reduction as
// (R, P_old), from which the neighbour warps form the new direction.
#pragma once
#include "common.cuh"

constexpr int kL64Warps = 8;
constexpr int kL64Threads = 32 * kL64Warps;

struct Geom64 {
    int w, h;             // subdomain extent (<= 64)
    int cp, r0;           // column pair and first row of the thread
    uint32_t um;          // bit 2k+j: pixel (row r0+k, column 2cp+j) is unknown and inside
    float nwl, nwr, nwu, nwd;   // -1 where that neighbour line lies in the subdomain, else 0
    float2 dh;            // horizontal part of d for the two columns
};

struct Shared64 {
    float2 msk[8][kL64Threads];               // 0/1 unknown-pixel mask per thread and row
    // [parity][boundary b between warps b and b+1][0: warp b's last row,
    // 1: warp b+1's first row][R, P_old][column pair]
    float2 seam[2][kL64Warps - 1][2][2][32];
    float red[5][kL64Warps];
};

__device__ __forceinline__ Geom64 make_geom64(int x0, int y0, int H, int W, const MaskView& m, Shared64& sh) {
    const int t = threadIdx.x, lane = t & 31, wv = t >> 5;
    Geom64 g;
    g.w = min(64, W - x0);
    g.h = min(64, H - y0);
    g.cp = lane;
    g.r0 = 8 * wv;
    const int c0 = 2 * lane;
    uint32_t um = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int R = g.r0 + k;
        // mask bits of the row at columns c0, c0 + 1 (rows past the subdomain read as known)
        uint32_t kn = 3u;
        if (R < g.h && c0 < g.w) kn = (m.window(x0 + (c0 & ~31), y0 + R) >> (c0 & 31)) & 3u;   // x < W: in bounds
        const bool u0 = c0 < g.w && R < g.h && !(kn & 1u), u1 = c0 + 1 < g.w && R < g.h && !(kn & 2u);
        um |= (u0 ? 1u : 0u) << (2 * k);
        um |= (u1 ? 1u : 0u) << (2 * k + 1);
        sh.msk[k][t] = make_float2(u0 ? 1.f : 0.f, u1 ? 1.f : 0.f);
    }
    g.um = um;
    auto horiz = [&](int C) { return ((C > 0) ? 1.f : 0.f) + ((C < g.w - 1) ? 1.f : 0.f); };
    g.dh = make_float2(horiz(c0), horiz(c0 + 1));
    g.nwl = (lane > 0) ? -1.f : 0.f;
    g.nwr = (lane < 31) ? -1.f : 0.f;
    g.nwu = (g.r0 > 0) ? -1.f : 0.f;
    g.nwd = (g.r0 + 8 < 64) ? -1.f : 0.f;
    return g;
}

__device__ __forceinline__ float2 diag64(const Geom64& g, int k) {
    const int R = g.r0 + k;
    const float v = ((R > 0) ? 1.f : 0.f) + ((R < g.h - 1) ? 1.f : 0.f);
    return make_float2(g.dh.x + v, g.dh.y + v);
}

__device__ __forceinline__ float cta_sum64(float v, Shared64& sh, int slot) {
    v = warp_sum_f(v);
    if ((threadIdx.x & 31) == 0) sh.red[slot][threadIdx.x >> 5] = v;
    __syncthreads();
    const float* r = sh.red[slot];
    return ((r[0] + r[1]) + (r[2] + r[3])) + ((r[4] + r[5]) + (r[6] + r[7]));
}

// Q = A_i P (P is zero on known and outside pixels).
__device__ __forceinline__ void apply64(const Geom64& g, const Shared64& sh, const float2 (&P)[8], float2 up,
                                        float2 dn, float2 (&Q)[8]) {
    const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float2 mk = sh.msk[k][threadIdx.x];
        const float L = __shfl_up_sync(HDI_FULL, P[k].y, 1);     // column 2cp-1
        const float Rt = __shfl_down_sync(HDI_FULL, P[k].x, 1);  // column 2cp+2
        float2 ns;
        ns.x = fmaf(g.nwl, L, -P[k].y);
        ns.y = fmaf(g.nwr, Rt, -P[k].x);
        if (k > 0) ns = __ffma2_rn(m1, P[k - 1], ns);
        else ns = __ffma2_rn(make_float2(g.nwu, g.nwu), up, ns);
        if (k < 7) ns = __ffma2_rn(m1, P[k + 1], ns);
        else ns = __ffma2_rn(make_float2(g.nwd, g.nwd), dn, ns);
        Q[k] = __ffma2_rn(mk, ns, __fmul2_rn(diag64(g, k), P[k]));
    }
}

// CG on A_i v = r from v = 0 (r: right-hand side in, residual out); stops
// when ||r||^2 <= thresh or after maxit iterations. All 256 threads call it.
__device__ __forceinline__ int cg64(const Geom64& g, Shared64& sh, float2 (&V)[8], float2 (&R)[8], float thresh,
                                    int maxit) {
    const int wv = threadIdx.x >> 5;
    const int c = g.cp;
    const bool wlast = wv < kL64Warps - 1, wfirst = wv > 0;   // writes side 0 of boundary wv / side 1 of wv - 1
    const int bup = wfirst ? wv - 1 : 0;                        // boundary above (clamped when absent)
    const int bdn = wlast ? wv : kL64Warps - 2;                 // boundary below
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
    if (wlast) { sh.seam[0][wv][0][0][c] = R[7]; sh.seam[0][wv][0][1][c] = z2; }
    if (wfirst) { sh.seam[0][wv - 1][1][0][c] = R[0]; sh.seam[0][wv - 1][1][1][c] = z2; }
    float rr = cta_sum64((a0.x + a0.y) + (a1.x + a1.y), sh, 4);
    float beta = 0.f;
    int it = 0;
    while (rr > thresh && it < maxit) {
        const int par = it & 1;
        const float2 b2 = make_float2(beta, beta);
        const float2 up = __ffma2_rn(b2, sh.seam[par][bup][0][1][c], sh.seam[par][bup][0][0][c]);
        const float2 dn = __ffma2_rn(b2, sh.seam[par][bdn][1][1][c], sh.seam[par][bdn][1][0][c]);
        apply64(g, sh, P, up, dn, Q);
        a0 = make_float2(0.f, 0.f);
        a1 = a0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (k & 1) a1 = __ffma2_rn(P[k], Q[k], a1);
            else a0 = __ffma2_rn(P[k], Q[k], a0);
        }
        const float pq = cta_sum64((a0.x + a0.y) + (a1.x + a1.y), sh, par * 2);
        if (!(pq > 0.f)) break;
        const float alpha = __fdividef(rr, pq);
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
        if (wlast) { sh.seam[npar][wv][0][0][c] = R[7]; sh.seam[npar][wv][0][1][c] = P[7]; }
        if (wfirst) { sh.seam[npar][wv - 1][1][0][c] = R[0]; sh.seam[npar][wv - 1][1][1][c] = P[0]; }
        const float rn = cta_sum64((a0.x + a0.y) + (a1.x + a1.y), sh, par * 2 + 1);
        beta = __fdividef(rn, rr);
        rr = rn;
        const float2 be = make_float2(beta, beta);
#pragma unroll
        for (int k = 0; k < 8; ++k) P[k] = __ffma2_rn(be, P[k], R[k]);
        ++it;
    }
    return it;
}

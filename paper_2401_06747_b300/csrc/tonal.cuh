// tonal.cuh -- tonal optimisation by restricted additive Schwarz on the
// normal equations (Sec. 5.2, Alg. 2).
//
//   1. r = B^T (f - B g): y = B g solves A y = C g; w solves A w = (I-C)(f-y)
//      (A~ acts on U as L_UU, Sec. 5.1); r_K = (f - y)_K + sum_{n in N(k) cap U} w_n.
//      Both solves are warm-started from the previous outer iteration
//      (Sec. 5.2, first paragraph after Alg. 2).
//   2. For every subdomain i (32x32, the ORAS tiling of level 0, or the
//      paper's 64x64, overlap 6 in both):
//      B_i^T B_i v_i = R_i r with B_i the subdomain's inpainting operator under
//      homogeneous Neumann conditions at the subdomain boundary (Sec. 5.2).
//   3. g <- g + sum_i R_i^T D_i v_i, D_i = 1 / multiplicity ("simple
//      averaging", Sec. 5.2).
//
// Local solves. The mask is fixed during tonal optimisation, so the local
// matrices B_i^T B_i = I + S_i^T S_i (S_i = L_UU,i^{-1} L_UK,i, in the mask
// pixel coordinates of the subdomain) are the same in every outer iteration.
// They are built once per call: S_i e_k (the negated local inpainting echo of
// mask pixel k) by CG on the Neumann subdomain problem (two warps per 32x32
// subdomain, eight per 64x64 one), the Gram matrix I + S^T S by a tiled
// product, its Cholesky factor and from it the explicit inverse. Each outer
// iteration then solves the local systems exactly by one dense symmetric
// matrix-vector product per subdomain instead of the paper's inner CGNR
// iterations.
#pragma once
#include "oras.cuh"
#include "anderson.cuh"
#include "cgnr.cuh"
#include "local64.cuh"

constexpr int kTonalMaxM = 4096;  // mask pixels per 64x64 subdomain (all of them)
constexpr int kGramSmem = 208;    // subdomains with more mask pixels factor G_i in global memory

// ----------------------------------------------------------- setup kernels ---

// Valid-column mask of a subdomain of width w (bits 0..w-1).
__device__ __forceinline__ uint32_t cols_valid(int w) { return w >= 32 ? 0xffffffffu : ((1u << w) - 1u); }

// Mask bits of row ly of a blk x blk subdomain (blk = 32 or 64), columns
// 32 * half .. 32 * half + 31 (zero outside the subdomain).
__device__ __forceinline__ uint32_t sub_row_bits(const MaskView& m, int x0, int y0, int w, int h, int ly, int half) {
    if (ly >= h || 32 * half >= w) return 0u;
    return m.window(x0 + 32 * half, y0 + ly) & cols_valid(w - 32 * half);
}

// m_i = number of mask pixels in subdomain i (warp per subdomain, lane = row).
__global__ void k_tonal_count(MaskView m, int nbx, int nby, int stride, int blk, int* __restrict__ cnt) {
    const int wid = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (wid >= nbx * nby) return;
    const int by = wid / nbx, bx = wid - by * nbx;
    const int x0 = sub_origin_n(bx, m.W, stride, blk), y0 = sub_origin_n(by, m.H, stride, blk);
    const int w = min(blk, m.W - x0), h = min(blk, m.H - y0);
    int c = 0;
    for (int ly = lane; ly < blk; ly += 32)
        for (int half = 0; half < blk / 32; ++half) c += __popc(sub_row_bits(m, x0, y0, w, h, ly, half));
    c = __reduce_add_sync(HDI_FULL, c);
    if (lane == 0) cnt[wid] = c;
}

// Local pixel codes (ly * blk + lx) of the mask pixels of each subdomain,
// in raster order, at list + off[i] (lane = row; rows 32.. in a second round).
__global__ void k_tonal_list(MaskView m, int nbx, int nby, int stride, int blk, const int* __restrict__ off,
                             uint16_t* __restrict__ list, int* __restrict__ owner) {
    const int wid = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (wid >= nbx * nby) return;
    const int by = wid / nbx, bx = wid - by * nbx;
    const int x0 = sub_origin_n(bx, m.W, stride, blk), y0 = sub_origin_n(by, m.H, stride, blk);
    const int w = min(blk, m.W - x0), h = min(blk, m.H - y0);
    int base = off[wid];
    for (int r0 = 0; r0 < blk; r0 += 32) {
        const int ly = r0 + lane;
        uint32_t bits[2] = {sub_row_bits(m, x0, y0, w, h, ly, 0), blk > 32 ? sub_row_bits(m, x0, y0, w, h, ly, 1) : 0u};
        const int c = __popc(bits[0]) + __popc(bits[1]);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(HDI_FULL, incl, o);
            if (lane >= o) incl += t;
        }
        int pos = base + incl - c;
        for (int half = 0; half < 2; ++half) {
            uint32_t b = bits[half];
            while (b) {
                const int lx = 32 * half + __ffs(b) - 1;
                b &= b - 1;
                owner[pos] = wid;
                list[pos++] = (uint16_t)(ly * blk + lx);
            }
        }
        base += __shfl_sync(HDI_FULL, incl, 31);
    }
}

struct EchoArgs {
    MaskView m;
    int nbx, nby, stride, nb;
    const int* off;          // [nb + 1] exclusive prefix of m_i
    const uint16_t* list;
    const int* owner;        // [sum m_i] subdomain of each echo
    float* echo;             // [sum m_i][blk rows][blk columns]
    float rtol2;
    int maxit;
    unsigned long long* iters;
};

// Right-hand side L_UK e_k of an echo solve at the lane's pixels: -1 at the
// unknown 4-neighbours of the mask pixel (kx, ky) inside the subdomain. The
// lane holds the column pair (c0, c0 + 1) over rows r0 .. r0 + NR - 1; um
// has bit 2k + j set where pixel (r0 + k, c0 + j) is unknown and inside.
template <int NR>
__device__ __forceinline__ void echo_rhs(int kx, int ky, int c0, int r0, uint32_t um, float2 (&R)[NR]) {
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int y = r0 + k;
        const bool nx = (c0 == kx && (y == ky - 1 || y == ky + 1)) || (y == ky && (c0 == kx - 1 || c0 == kx + 1));
        const bool ny =
            (c0 + 1 == kx && (y == ky - 1 || y == ky + 1)) || (y == ky && (c0 + 1 == kx - 1 || c0 + 1 == kx + 1));
        R[k].x = (nx && ((um >> (2 * k)) & 1u)) ? -1.f : 0.f;
        R[k].y = (ny && ((um >> (2 * k + 1)) & 1u)) ? -1.f : 0.f;
    }
}

// One warp per (subdomain, mask pixel k), in the layout of the one-warp ORAS
// sweep (oras_warp.cuh: lane = column pair x 16 rows, dot products by warp
// butterflies, no barriers): solve the Neumann subdomain problem
// L_UU x = L_UK e_k by CG (theta = 0 at every subdomain side) to
// ||r|| <= rtol ||L_UK e_k||; x = S e_k is stored row-major over the 32x32
// tile (zero on known and outside pixels). FULL: every subdomain is 32x32
// (images of at least 32 x 32 pixels).
template <bool FULL>
__global__ void __launch_bounds__(32, 12) k_tonal_echo_w(EchoArgs a) {
    __shared__ WarpShared sh;
    const long long e = blockIdx.x;
    if (e >= a.off[a.nb]) return;   // the whole warp (the CTA) leaves together
    const int i = a.owner[e];
    const int by = i / a.nbx, bx = i - by * a.nbx;
    const int x0 = sub_origin(bx, a.m.W, a.stride), y0 = sub_origin(by, a.m.H, a.stride);
    const WarpGeom g = make_wgeom(x0, y0, a.m.H, a.m.W, a.m, 0.f, sh);
    const int code = a.list[e];
    const int c0 = 2 * g.c, r0 = g.r0;
    float2 R[kWarpRows], V[kWarpRows];
    echo_rhs(code & 31, code >> 5, c0, r0, g.um, R);
    const float rr0 = warp_sum_f(wdot(R, R));
    __syncwarp();   // the mask floats of make_wgeom are read by the same lanes only
    const int it = warp_cg<FULL>(g, sh, V, R, a.rtol2 * rr0, a.maxit);
    if (a.iters && (threadIdx.x & 31) == 0 && it) atomicAdd(a.iters, (unsigned long long)it);
    float* out = a.echo + (size_t)e * 1024;
#pragma unroll
    for (int k = 0; k < kWarpRows; ++k) *reinterpret_cast<float2*>(out + (r0 + k) * 32 + c0) = V[k];
}

// One CTA (two warps) per (subdomain, mask pixel k): the same echo solve in
// the two-warp layout of k_oras (oras_warp = 0).
__global__ void __launch_bounds__(kLocalThreads, 8) k_tonal_echo(EchoArgs a) {
    __shared__ LocalShared sh;
    const long long e = blockIdx.x;
    const int total = a.off[a.nb];
    if (e >= total) return;
    const int i = a.owner[e];
    const int by = i / a.nbx, bx = i - by * a.nbx;
    const int x0 = sub_origin(bx, a.m.W, a.stride), y0 = sub_origin(by, a.m.H, a.stride);
    const LocalGeom g = make_geom(x0, y0, a.m.H, a.m.W, a.m, 0.f, sh);
    const int code = a.list[e];
    const int ky = code >> 5, kx = code & 31;
    const int c0 = 2 * g.c, r0 = g.r0;
    // right-hand side L_UK e_k: -1 at the unknown 4-neighbours of k inside the subdomain
    float2 R[8], V[8];
    float2 a0 = make_float2(0.f, 0.f);
    echo_rhs(kx, ky, c0, r0, g.um, R);
#pragma unroll
    for (int k = 0; k < 8; ++k) a0 = __ffma2_rn(R[k], R[k], a0);
    const float rr0 = cta_sum2(a0.x + a0.y, sh, 3);   // slot 4 is reused right away by the CG set-up
    const int it = (g.w == 32 && g.h == 32) ? local_cg<true>(g, sh, V, R, a.rtol2 * rr0, a.maxit)
                                            : local_cg<false>(g, sh, V, R, a.rtol2 * rr0, a.maxit);
    if (a.iters && threadIdx.x == 0 && it) atomicAdd(a.iters, (unsigned long long)it);
    float* out = a.echo + (size_t)e * 1024;
#pragma unroll
    for (int k = 0; k < 8; ++k) *reinterpret_cast<float2*>(out + (r0 + k) * 32 + c0) = V[k];
}

// The same on 64x64 subdomains: one CTA of eight warps per (subdomain, mask
// pixel k); x = S e_k stored row-major over the 64x64 tile.
__global__ void __launch_bounds__(kL64Threads, 2) k_tonal_echo64(EchoArgs a) {
    __shared__ Shared64 sh;
    const long long e = blockIdx.x;
    const int total = a.off[a.nb];
    if (e >= total) return;
    const int i = a.owner[e];
    const int by = i / a.nbx, bx = i - by * a.nbx;
    const int x0 = sub_origin_n(bx, a.m.W, a.stride, 64), y0 = sub_origin_n(by, a.m.H, a.stride, 64);
    const Geom64 g = make_geom64(x0, y0, a.m.H, a.m.W, a.m, sh);
    const int code = a.list[e];
    const int ky = code >> 6, kx = code & 63;
    const int c0 = 2 * g.cp, r0 = g.r0;
    float2 R[8], V[8];
    float2 a0 = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int y = r0 + k;
        const bool nx = (c0 == kx && (y == ky - 1 || y == ky + 1)) || (y == ky && (c0 == kx - 1 || c0 == kx + 1));
        const bool ny =
            (c0 + 1 == kx && (y == ky - 1 || y == ky + 1)) || (y == ky && (c0 + 1 == kx - 1 || c0 + 1 == kx + 1));
        R[k].x = (nx && ((g.um >> (2 * k)) & 1u)) ? -1.f : 0.f;
        R[k].y = (ny && ((g.um >> (2 * k + 1)) & 1u)) ? -1.f : 0.f;
        a0 = __ffma2_rn(R[k], R[k], a0);
    }
    const float rr0 = cta_sum64(a0.x + a0.y, sh, 3);
    const int it = cg64(g, sh, V, R, a.rtol2 * rr0, a.maxit);
    if (a.iters && threadIdx.x == 0 && it) atomicAdd(a.iters, (unsigned long long)it);
    float* out = a.echo + (size_t)e * 4096;
#pragma unroll
    for (int k = 0; k < 8; ++k) *reinterpret_cast<float2*>(out + (r0 + k) * 64 + c0) = V[k];
}


// Shared-memory floats of k_tonal_gram for subdomains of up to m mask pixels.
__host__ __device__ inline int gram_round4(int m) { return (m + 3) & ~3; }
// The staged pixels and the partial blocks of the sliced product share one
// region (the partial blocks are written after the last staged round).
__host__ __device__ inline size_t gram_stage_floats(int m4) {
    return (size_t)32 * (m4 + 4) > 256 * 16 ? (size_t)32 * (m4 + 4) : (size_t)256 * 16;
}
__host__ __device__ inline size_t gram_smem_floats(int m) {
    const int m4 = gram_round4(m);
    return (size_t)m * (m | 1) + 4 + gram_stage_floats(m4) + m4;
}

// G_i = I + S_i^T S_i and its inverse (full m x m, row-major) at
// fac + goff[i]. One CTA of 256 threads per subdomain.
// Products: each thread accumulates one 4x4 block of the lower triangle of G
// (m rounded up to a multiple of 4); with few blocks the npx pixels are
// split into ks interleaved slices whose partial blocks are added in a fixed
// order. Pixels are staged 32 at a time in shared memory, transposed, so a
// thread reads four echoes' values of one pixel with one 16-byte load.
// Cholesky (right-looking): thread r owns row r, two barriers per column.
// Inverse: W = L^{-1} column by column (thread j forward-substitutes e_j;
// W^T is kept in the free upper triangle of G's buffer), then
// G^{-1} = W^T W, written in full so the local solves are one dense
// symmetric matrix-vector product.
__global__ void __launch_bounds__(256) k_tonal_gram(const int* __restrict__ off, const long long* __restrict__ goff,
                                                    const float* __restrict__ echo, float* __restrict__ fac,
                                                    unsigned* bad, int npx) {
    extern __shared__ __align__(16) float sm[];
    const int i = blockIdx.x;
    const int m = off[i + 1] - off[i];
    if (m == 0 || m > kGramSmem) return;   // dense subdomains: k_tonal_gram_big
    const int tid = threadIdx.x;
    const int m4 = gram_round4(m);
    const int nb = m4 / 4;
    const int nblk = nb * (nb + 1) / 2;
    const int ks = (nblk >= 256) ? 1 : min(8, 256 / nblk);
    const int gs = m | 1;                          // row stride of G
    const int es = m4 + 4;                         // row stride of the staged pixels
    float* G = sm;                                 // m x gs
    float* Es = sm + (((size_t)m * gs + 3) & ~(size_t)3);   // [32][es], 16-byte aligned rows
    float* part = Es;                              // [ks][nblk][16] (ks > 1), after the last staged round
    const float* E = echo + (size_t)off[i] * npx;
    for (int b0 = 0; b0 < nblk; b0 += 256) {       // rounds of up to 256 blocks (ks == 1 when > 1 round)
        const int slot = tid % (ks > 1 ? nblk : 256);
        const int sl = tid / (ks > 1 ? nblk : 256);
        const int bidx = b0 + slot;
        const bool on = sl < ks && bidx < nblk && (ks == 1 || slot < nblk);
        int br = 0, bc = 0;
        if (on) {
            br = (int)((sqrtf(8.f * (float)bidx + 1.f) - 1.f) * 0.5f);
            while (br * (br + 1) / 2 > bidx) --br;
            while ((br + 1) * (br + 2) / 2 <= bidx) ++br;
            bc = bidx - br * (br + 1) / 2;
        }
        float acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
        for (int p0 = 0; p0 < npx; p0 += 32) {
            __syncthreads();
            for (int q = tid; q < m4 * 32; q += 256) {
                const int k = q >> 5, pp = q & 31;
                Es[pp * es + k] = (k < m) ? E[(size_t)k * npx + p0 + pp] : 0.f;
            }
            __syncthreads();
            if (on) {
                for (int pp = sl; pp < 32; pp += ks) {
                    const float4 av = *reinterpret_cast<const float4*>(Es + pp * es + 4 * br);
                    const float4 bv = *reinterpret_cast<const float4*>(Es + pp * es + 4 * bc);
                    const float a4[4] = {av.x, av.y, av.z, av.w}, b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(a4[a], b4[b], acc[a][b]);
                }
            }
        }
        if (ks > 1) {
            __syncthreads();   // every thread is done reading the staged pixels that part overwrites
            if (on) {
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) part[((size_t)sl * nblk + slot) * 16 + a * 4 + b] = acc[a][b];
            }
            __syncthreads();
            if (tid < nblk) {
                for (int e = 0; e < 16; ++e) {
                    float t = part[(size_t)tid * 16 + e];
                    for (int q = 1; q < ks; ++q) t += part[((size_t)q * nblk + tid) * 16 + e];
                    acc[e >> 2][e & 3] = t;
                }
            }
        }
        const bool own = (ks > 1) ? (tid < nblk) : on;
        if (own) {
            if (ks > 1) {   // the summing thread tid holds block tid
                br = (int)((sqrtf(8.f * (float)tid + 1.f) - 1.f) * 0.5f);
                while (br * (br + 1) / 2 > tid) --br;
                while ((br + 1) * (br + 2) / 2 <= tid) ++br;
                bc = tid - br * (br + 1) / 2;
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int r = 4 * br + a, c = 4 * bc + b;
                    if (r < m && c <= r) G[r * gs + c] = acc[a][b] + (r == c ? 1.f : 0.f);
                }
        }
    }
    __syncthreads();
    // G = Lu D Lu^T (Lu unit lower triangular) by right-looking elimination:
    // step j subtracts u_rj u_cj / d_j from the trailing entries j < c <= r
    // (u: the column below the pivot d_j = G[j][j], kept unscaled). The
    // trailing triangle is spread over a 16 x 16 grid of threads, so a step
    // costs O((m - j)^2 / 256) per thread and one barrier; a step reads only
    // column j and writes only columns after it.
    const int tr = tid >> 4, tc = tid & 15;
    for (int j = 0; j + 1 < m; ++j) {
        const float pinv = 1.f / G[j * gs + j];
        for (int r = j + 1 + tr; r < m; r += 16) {
            const float ur = G[r * gs + j] * pinv;
            for (int c = j + 1 + tc; c <= r; c += 16) G[r * gs + c] = fmaf(-ur, G[c * gs + j], G[r * gs + c]);
        }
        __syncthreads();
    }
    // Lu below the diagonal (u / d), 1 / d in dinv, the upper triangle
    // cleared for V^T. Every pivot of the SPD G is positive.
    float* dinv = Es + gram_stage_floats(m4);
    for (int r = tr; r < m; r += 16) {
        const float dr = G[r * gs + r];
        for (int c = tc; c < m; c += 16) {
            if (c < r) G[r * gs + c] = G[r * gs + c] / G[c * gs + c];
            else if (c > r) G[r * gs + c] = 0.f;
        }
        if (tc == 0) {
            if (!(dr > 0.f)) atomicOr(bad, 1u);
            dinv[r] = 1.f / dr;
        }
    }
    __syncthreads();
    // V = Lu^{-1} (unit lower triangular) by forward elimination on I:
    // step k subtracts Lu[q][k] row_k(V) from the rows q > k (row k of V is
    // final after step k - 1; its diagonal is 1). V[q][j], q > j, is kept
    // transposed in the upper triangle, at G[j][q]; a step reads column k
    // of both triangles and writes columns q > k of the upper one.
    for (int k = 0; k + 1 < m; ++k) {
        for (int q = k + 1 + tr; q < m; q += 16) {   // row q of V (i is the subdomain)
            const float l = G[q * gs + k];
            for (int j = tc; j <= k; j += 16) {
                const float vkj = (j == k) ? 1.f : G[j * gs + k];
                G[j * gs + q] = fmaf(-l, vkj, G[j * gs + q]);
            }
        }
        __syncthreads();
    }
    // G^{-1} = V^T D^{-1} V: [a][b] = sum_{k >= max(a, b)} V[k][a] V[k][b] / d_k,
    // entries a >= b (V[k][a] = G[a][k] for k > a, V[a][a] = 1)
    float* Gi = fac + goff[i];
    const int ne = m * (m + 1) / 2;
    for (int e = tid; e < ne; e += 256) {
        int ra = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
        while (ra * (ra + 1) / 2 > e) --ra;
        while ((ra + 1) * (ra + 2) / 2 <= e) ++ra;
        const int cb = e - ra * (ra + 1) / 2;
        // k = ra term: V[ra][ra] V[ra][cb] / d_ra (V[ra][cb] = G[cb][ra], or 1 when cb == ra)
        float acc = dinv[ra] * ((cb == ra) ? 1.f : G[cb * gs + ra]);
        for (int k = ra + 1; k < m; ++k) acc = fmaf(G[ra * gs + k] * dinv[k], G[cb * gs + k], acc);
        Gi[(size_t)ra * m + cb] = acc;
        Gi[(size_t)cb * m + ra] = acc;
    }
}

// Dense subdomains (m_i > kGramSmem mask pixels): the same G_i and inverse,
// with G_i in its global output block instead of shared memory. The Gram
// product uses the same register blocks (pixels staged in shared memory); the
// Cholesky factor and W = L^{-1} (as W^T in the upper triangle) are formed
// in place, G_i^{-1} = W^T W is written to the subdomain's echo block, which
// the product no longer needs (m_i x npx >= m_i x m_i floats), and copied
// back. Threads own rows r = tid, tid + 256, ...
__global__ void __launch_bounds__(256) k_tonal_gram_big(const int* __restrict__ off,
                                                        const long long* __restrict__ goff,
                                                        float* __restrict__ echo, float* __restrict__ fac,
                                                        unsigned* bad, int npx) {
    extern __shared__ __align__(16) float sm[];
    const int i = blockIdx.x;
    const int m = off[i + 1] - off[i];
    if (m <= kGramSmem) return;
    const int tid = threadIdx.x;
    const int m4 = gram_round4(m);
    const int nb = m4 / 4;
    const long long nblk = (long long)nb * (nb + 1) / 2;
    const int es = m4 + 4;
    float* Es = sm;                        // [32][es]
    float* dinv = sm + 32 * es;            // [m]
    float* col = dinv + m4;                // [m]: the current column of L
    float* sd = col + m4;                  // [1]: the current diagonal
    float* G = fac + goff[i];              // m x m
    float* E = echo + (size_t)off[i] * npx;
    // G = I + S^T S, lower triangle, 4x4 blocks
    for (long long b0 = 0; b0 < nblk; b0 += 256) {
        const long long bidx = b0 + tid;
        const bool on = bidx < nblk;
        int br = 0, bc = 0;
        if (on) {
            br = (int)((sqrtf(8.f * (float)bidx + 1.f) - 1.f) * 0.5f);
            while ((long long)br * (br + 1) / 2 > bidx) --br;
            while ((long long)(br + 1) * (br + 2) / 2 <= bidx) ++br;
            bc = (int)(bidx - (long long)br * (br + 1) / 2);
        }
        float acc[4][4];
#pragma unroll
        for (int aa = 0; aa < 4; ++aa)
#pragma unroll
            for (int bb = 0; bb < 4; ++bb) acc[aa][bb] = 0.f;
        for (int p0 = 0; p0 < npx; p0 += 32) {
            __syncthreads();
            for (int q = tid; q < m4 * 32; q += 256) {
                const int k = q >> 5, pp = q & 31;
                Es[pp * es + k] = (k < m) ? E[(size_t)k * npx + p0 + pp] : 0.f;
            }
            __syncthreads();
            if (on) {
                for (int pp = 0; pp < 32; ++pp) {
                    const float4 av = *reinterpret_cast<const float4*>(Es + pp * es + 4 * br);
                    const float4 bv = *reinterpret_cast<const float4*>(Es + pp * es + 4 * bc);
                    const float a4[4] = {av.x, av.y, av.z, av.w}, b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                    for (int aa = 0; aa < 4; ++aa)
#pragma unroll
                        for (int bb = 0; bb < 4; ++bb) acc[aa][bb] = fmaf(a4[aa], b4[bb], acc[aa][bb]);
                }
            }
        }
        if (on) {
#pragma unroll
            for (int aa = 0; aa < 4; ++aa)
#pragma unroll
                for (int bb = 0; bb < 4; ++bb) {
                    const int r = 4 * br + aa, c = 4 * bc + bb;
                    if (r < m && c <= r) G[(size_t)r * m + c] = acc[aa][bb] + (r == c ? 1.f : 0.f);
                }
        }
    }
    __syncthreads();
    // right-looking Cholesky in place (lower triangle)
    for (int j = 0; j < m; ++j) {
        if (tid == (j & 255)) {
            const float d = sqrtf(G[(size_t)j * m + j]);
            if (!(d > 0.f)) atomicOr(bad, 1u);
            G[(size_t)j * m + j] = d;
            sd[0] = d;
        }
        __syncthreads();
        const float dj = sd[0];
        for (int r = j + 1 + ((tid - j - 1) & 255); r < m; r += 256) {
            const float l = G[(size_t)r * m + j] / dj;
            G[(size_t)r * m + j] = l;
            col[r] = l;   // column j of L, read by every row's update
        }
        __syncthreads();
        for (int r = j + 1 + ((tid - j - 1) & 255); r < m; r += 256) {
            const float l = col[r];
            float* __restrict__ gr = G + (size_t)r * m;
            for (int c = j + 1; c <= r; ++c) gr[c] = fmaf(-l, col[c], gr[c]);
        }
        __syncthreads();
    }
    // W = L^{-1}: thread owns columns j; W^T row j in the upper triangle
    for (int r = tid; r < m; r += 256) {
        const float dj = 1.f / G[(size_t)r * m + r];
        dinv[r] = dj;
        for (int ii = r + 1; ii < m; ++ii) {
            const float* li = G + (size_t)ii * m;
            float s0 = li[r] * dj, s1 = 0.f;
            int k = r + 1;
            for (; k + 1 < ii; k += 2) {
                s0 = fmaf(li[k], G[(size_t)r * m + k], s0);
                s1 = fmaf(li[k + 1], G[(size_t)r * m + k + 1], s1);
            }
            if (k < ii) s0 = fmaf(li[k], G[(size_t)r * m + k], s0);
            G[(size_t)r * m + ii] = -(s0 + s1) / li[ii];
        }
    }
    __syncthreads();
    // G^{-1} = W^T W into the echo block, then back
    const long long ne = (long long)m * (m + 1) / 2;
    for (long long e = tid; e < ne; e += 256) {
        int ra = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
        while ((long long)ra * (ra + 1) / 2 > e) --ra;
        while ((long long)(ra + 1) * (ra + 2) / 2 <= e) ++ra;
        const int cb = (int)(e - (long long)ra * (ra + 1) / 2);
        float acc = dinv[ra] * ((cb == ra) ? dinv[ra] : G[(size_t)cb * m + ra]);
        for (int k = ra + 1; k < m; ++k) acc = fmaf(G[(size_t)ra * m + k], G[(size_t)cb * m + k], acc);
        E[(size_t)ra * m + cb] = acc;
        E[(size_t)cb * m + ra] = acc;
    }
    __syncthreads();
    for (long long e = tid; e < (long long)m * m; e += 256) G[e] = E[e];
}

// ------------------------------------------------------- outer iteration ---

// B^T (f - y) on the mask pixels, from the list of mask pixels (raster order,
// level-0 offsets y * pitch + x): r_K = (f - y)_K + sum of w over the unknown
// in-image 4-neighbours (Sec. 5.1), in double-float, written to r at the
// pixel; per channel ||r_K||^2 into red_r and ||(f - y)_K||^2 into red_e (the
// unknown pixels' part of ||f - y||^2 is the right-hand-side norm of the
// adjoint solve). y == nullptr means y = 0. One pass over the list per
// channel (grid y), a thread per mask pixel.
__global__ void __launch_bounds__(256) k_tonal_residual(LevelArr F, MaskView m, DFc f, DFc y, DFc w,
                                                        const int* __restrict__ list, int M, float* __restrict__ r,
                                                        GridReduce red_r, GridReduce red_e) {
    const int ch = blockIdx.y;
    const size_t co = (size_t)ch * F.cs;
    float se = 0.f, sr = 0.f;
    for (int i = blockIdx.x * 256 + threadIdx.x; i < M; i += gridDim.x * 256) {
        const int p = list[i];
        const int py = p / F.pitch, px = p - py * F.pitch;
        const size_t at = co + p;
        float sh = f.hi[at], sl = f.lo[at];
        if (y.hi) df_add(sh, sl, -y.hi[at], -y.lo[at], sh, sl);
        se += (sh + sl) * (sh + sl);
        float ah = sh, al = sl;
        const bool nb[4] = {px > 0 && !m.known(px - 1, py), px + 1 < F.W && !m.known(px + 1, py),
                            py > 0 && !m.known(px, py - 1), py + 1 < F.H && !m.known(px, py + 1)};
        const long long off[4] = {-1, 1, -(long long)F.pitch, (long long)F.pitch};
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (nb[q]) df_add(ah, al, w.hi[at + off[q]], w.lo[at + off[q]], ah, al);
        const float rv = ah + al;
        r[at] = rv;
        sr += rv * rv;
    }
    const double tr = (double)block_sum_f(sr);
    grid_reduce_commit(red_r, ch, blockIdx.x, tr);
    const double te = (double)block_sum_f(se);
    grid_reduce_commit(red_e, ch, blockIdx.x, te);
}

struct LocalSolveArgs {
    LevelArr F;
    int nbx, nby, stride, nch, color;
    int blk, lb;             // subdomain side (32 or 64) and its log2
    const int* off;
    const long long* goff;
    const uint16_t* list;
    const float* fac;
    const float* r;
    float* out;      // full layout, accumulates D_i v_i (zeroed before the first colour)
};

// Number of subdomains covering coordinate x along an axis of n pixels
// (1 or 2; the last subdomain sits at sub_origin(nb - 1, n, stride)).
__device__ __forceinline__ int cover_count(int x, int nb, int stride, int n, int blk) {
    if (nb == 1) return 1;
    const int hi = min(nb - 2, x / stride);
    const int lo = max(0, (x - (blk - 1) + stride - 1) / stride);
    int c = (hi >= lo) ? hi - lo + 1 : 0;
    if (x >= sub_origin_n(nb - 1, n, stride, blk)) ++c;
    return c;
}

// Colour classes along one axis: the last subdomain (which sits at the
// border and may overlap the one two places earlier) is class 2, the others
// alternate 0, 1. Two subdomains of one class never overlap.
__host__ __device__ __forceinline__ int class_count(int c, int nb) {
    const int inner = (nb >= 2) ? nb - 1 : nb;
    if (c == 2) return (nb >= 2) ? 1 : 0;
    return (inner - c + 1) / 2;
}
__host__ __device__ __forceinline__ int class_member(int c, int q, int nb) { return c == 2 ? nb - 1 : c + 2 * q; }

// Local solves of one colour class (cx, cy), color = cy * 3 + cx:
// v = G_i^{-1} R_i r with the dense inverse from the setup, then
// out += D_i v (out = P r after all nine classes). Subdomains of one class
// never overlap, so the updates need no atomics and their order is fixed.
// One CTA of kLocalWarps warps per subdomain solves all channels: warp w
// takes the rows j = w, w + kLocalWarps, ... of the symmetric inverse (each
// read coalesced), lane l accumulates entries l, l + 32, ... of v, and the
// warps' partial sums are added in a fixed order.
constexpr int kLocalWarps = 4;
__global__ void __launch_bounds__(32 * kLocalWarps) k_tonal_local(LocalSolveArgs a) {
    constexpr int NT = 4;                 // rows of v per lane and pass: 128 per pass
    extern __shared__ float xs[];   // [4][m]: the channels' r at the mask pixels
    __shared__ float ps[kLocalWarps][4][NT * 32];
    // Only the final accumulation into `out` depends on the previous colour's
    // launch (r and the factors were complete before the colours started), so
    // the products run while that launch finishes; pdl_wait() guards the
    // writes.
    pdl_trigger();
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int cx = a.color % 3, cy = a.color / 3;
    const int hx = class_count(cx, a.nbx);
    const int hy = class_count(cy, a.nby);
    const int q = blockIdx.x;
    if (q >= hx * hy) return;
    const int bx = class_member(cx, q % hx, a.nbx);
    const int by = class_member(cy, q / hx, a.nby);
    const int i = by * a.nbx + bx;
    const int m = a.off[i + 1] - a.off[i];
    if (m == 0) return;
    const int nch = a.nch;   // 1..4 (image channels)
    const uint16_t* lst = a.list + a.off[i];
    const float* __restrict__ Gi = a.fac + a.goff[i];
    const int x0 = sub_origin_n(bx, a.F.W, a.stride, a.blk), y0 = sub_origin_n(by, a.F.H, a.stride, a.blk);
    auto pixel = [&](int k) {
        const int code = lst[k];
        return (size_t)(y0 + (code >> a.lb)) * a.F.pitch + x0 + (code & (a.blk - 1));
    };
    for (int k = threadIdx.x; k < m; k += 32 * kLocalWarps) {
        const size_t p = pixel(k);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (c < nch) xs[c * m + k] = a.r[c * a.F.cs + p];
    }
    __syncthreads();
    // passes over 128 rows of v (one pass unless the subdomain is dense)
    for (int base = 0; base < m; base += NT * 32) {
        float y[4][NT];
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int t = 0; t < NT; ++t) y[c][t] = 0.f;
#pragma unroll 4
        for (int j = wl; j < m; j += kLocalWarps) {
            const float* row = Gi + (size_t)j * m + base;
            float xj[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) xj[c] = (c < nch) ? xs[c * m + j] : 0.f;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const int k = lane + 32 * t;
                if (base + k < m) {
                    const float g = row[k];
#pragma unroll
                    for (int c = 0; c < 4; ++c) y[c][t] = fmaf(g, xj[c], y[c][t]);
                }
            }
        }
        if (base > 0) __syncthreads();   // the previous pass has read ps
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int t = 0; t < NT; ++t) ps[wl][c][t * 32 + lane] = y[c][t];
        pdl_wait();
        __syncthreads();
        for (int k = threadIdx.x; k < NT * 32 && base + k < m; k += 32 * kLocalWarps) {
            const int code = lst[base + k];
            const int px = x0 + (code & (a.blk - 1)), py = y0 + (code >> a.lb);
            const int mult =
                cover_count(px, a.nbx, a.stride, a.F.W, a.blk) * cover_count(py, a.nby, a.stride, a.F.H, a.blk);
            const size_t p = (size_t)py * a.F.pitch + px;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (c < nch) {
                    float v = ps[0][c][k];
#pragma unroll
                    for (int w = 1; w < kLocalWarps; ++w) v += ps[w][c][k];
                    a.out[c * a.F.cs + p] += v / (float)mult;
                }
            }
        }
    }
}


// ------------------------------------------------------- host-side loop ---

int Ctx::tonal_setup() {
    // RAS subdomain side: 64 (the paper's block) couples the subdomains
    // better at sparse masks, 32 keeps the local factors cheap at denser ones
    // (measured crossover between 2% and 4% at 4K)
    const double density = (double)mlist_n / ((double)H * W);
    const int blk = (p.tonal_block >= 48) ? 64 : (p.tonal_block >= 16 ? 32 : (density < 0.03 ? 64 : 32));
    int rc = tonal_setup_blk(blk);
    // a 64x64 block with more than 1024 mask pixels (a densely known region)
    // would need an m x m factorisation of up to 4096^2 in one CTA: such masks
    // take the 32x32 blocks instead
    if (rc == HDI_OK && blk == 64 && t_maxm > 1024) rc = tonal_setup_blk(32);
    return rc;
}

// Dynamic shared memory of k_tonal_gram_big for m mask pixels.
static inline size_t gram_big_smem_bytes(int m) {
    return ((size_t)32 * (gram_round4(m) + 4) + 2 * gram_round4(m) + 4) * 4;
}

// The Gram kernels' dynamic shared memory limits, set once per device at
// the largest size any call can launch with (m <= kGramSmem for
// k_tonal_gram, m <= 1024 mask pixels per subdomain for k_tonal_gram_big).
// The limit is a property of the function shared by every context and
// thread of the process: setting it per call to the call's own size let a
// concurrent call on another stream lower it between another call's setting
// and its launch. A launch's own size still sets its occupancy.
static void tonal_smem_limits(int device) {
    static std::once_flag once[64];
    if (device < 0 || device >= 64) return;
    std::call_once(once[device], [] {
        cudaFuncSetAttribute(k_tonal_gram, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(gram_smem_floats(kGramSmem) * 4));
        cudaFuncSetAttribute(k_tonal_gram_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)gram_big_smem_bytes(1024));
    });
}

int Ctx::tonal_setup_blk(int blk) {
    int rc;
    const int npx = blk * blk;
    const int stride = blk - kOv;
    t_blk = blk;
    t_nbx = tile_count(W, blk, kOv);
    t_nby = tile_count(H, blk, kOv);
    const int nb = t_nbx * t_nby;
    // counts
    std::vector<int> cnt(nb), off(nb + 1);
    std::vector<long long> goff(nb + 1);
    int* dcnt = nullptr;
    const int ncnt = std::max(nb, H) + 1;
    if ((rc = tws.reserve(*this, std::max(tws.cap, (size_t)ncnt * 24 + 4096), "tonal counts"))) return rc;
    dcnt = (int*)tws.take((size_t)ncnt * 4);
    k_tonal_count<<<(nb + 3) / 4, 128, 0, stream>>>(mview(0), t_nbx, t_nby, stride, blk, dcnt);
    ++launches;
    cudaMemcpyAsync(cnt.data(), dcnt, (size_t)nb * 4, cudaMemcpyDeviceToHost, stream);
    if ((rc = sync("tonal subdomain counts"))) return rc;
    off[0] = 0;
    goff[0] = 0;
    int maxm = 0;
    for (int i = 0; i < nb; ++i) {
        off[i + 1] = off[i] + cnt[i];
        goff[i + 1] = goff[i] + (long long)cnt[i] * cnt[i];
        maxm = std::max(maxm, cnt[i]);
    }
    t_maxm = maxm;
    if (blk == 64 && maxm > 1024) return HDI_OK;   // the caller retries with 32x32 blocks
    const long long total = off[nb];
    const int M = mlist_n;   // the mask list (built by the caller)
    const int mwin = (int)p.tonal_anderson;
    // layout
    size_t bytes = 0;
    auto acc = [&](size_t b) { bytes += (b + 255) & ~(size_t)255; };
    acc((size_t)nch * M * 4);
    acc((size_t)nch * M * 4);
    acc((size_t)std::max(mwin, 1) * nch * M * 4);
    acc((size_t)std::max(mwin, 1) * nch * M * 4);
    acc((size_t)nch * 64 * kAAParts * 8);
    acc((size_t)4 * 64 * 8);
    acc((size_t)4 * kAAMax * 8);
    acc(256);
    acc((size_t)(nb + 1) * 4);
    acc((size_t)(nb + 1) * 8);
    acc((size_t)total * 2);
    acc((size_t)total * 4);
    acc((size_t)total * npx * 4);
    acc((size_t)goff[nb] * 4);
    if ((rc = tws.reserve(*this, bytes, "tonal local factors"))) return rc;
    t_off = (int*)tws.take((size_t)(nb + 1) * 4);
    t_goff = (long long*)tws.take((size_t)(nb + 1) * 8);
    t_list = (uint16_t*)tws.take((size_t)total * 2);
    int* t_owner = (int*)tws.take((size_t)total * 4);
    t_echo = (float*)tws.take((size_t)total * npx * 4);
    t_fac = (float*)tws.take((size_t)goff[nb] * 4);
    aa_idx = mlist;
    aa_fv = (float*)tws.take((size_t)nch * M * 4);
    aa_fvprev = (float*)tws.take((size_t)nch * M * 4);
    aa_dF = (float*)tws.take((size_t)std::max(mwin, 1) * nch * M * 4);
    aa_dX = (float*)tws.take((size_t)std::max(mwin, 1) * nch * M * 4);
    aa_part = (double*)tws.take((size_t)nch * 64 * kAAParts * 8);
    aa_out = (double*)tws.take((size_t)4 * 64 * 8);
    aa_gam = (double*)tws.take((size_t)4 * kAAMax * 8);
    aa_ticket = (unsigned*)tws.take(256);
    if (tws.used > tws.cap) return fail(HDI_ERR_CUDA, "internal: tonal workspace carving exceeds its reservation");
    cudaMemsetAsync(aa_ticket, 0, 256, stream);
    aa_M = M;
    cudaMemcpyAsync(t_off, off.data(), (size_t)(nb + 1) * 4, cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(t_goff, goff.data(), (size_t)(nb + 1) * 8, cudaMemcpyHostToDevice, stream);
    k_tonal_list<<<(nb + 3) / 4, 128, 0, stream>>>(mview(0), t_nbx, t_nby, stride, blk, t_off, t_list, t_owner);
    ++launches;
    if (total > 0) {
        EchoArgs ea;
        ea.m = mview(0);
        ea.nbx = t_nbx;
        ea.nby = t_nby;
        ea.stride = stride;
        ea.nb = nb;
        ea.off = t_off;
        ea.list = t_list;
        ea.owner = t_owner;
        ea.echo = t_echo;
        ea.rtol2 = (float)(p.tonal_echo_rtol * p.tonal_echo_rtol);
        ea.maxit = (int)p.tonal_echo_max_iter;
        ea.iters = counters + kCntEcho;
        if (pending_upload) {   // Ctx::tonal's host f: copied while the echo and Gram kernels run
            const hdi_image* im = pending_upload;
            pending_upload = nullptr;
            if ((rc = upload_begin(im))) return rc;
        }
        tstart(kT_Echo);
        if (blk == 64) k_tonal_echo64<<<(unsigned)total, kL64Threads, 0, stream>>>(ea);
        else if (p.oras_warp >= 0.5 && W >= 32 && H >= 32)
            k_tonal_echo_w<true><<<(unsigned)total, 32, 0, stream>>>(ea);
        else if (p.oras_warp >= 0.5)
            k_tonal_echo_w<false><<<(unsigned)total, 32, 0, stream>>>(ea);
        else k_tonal_echo<<<(unsigned)total, kLocalThreads, 0, stream>>>(ea);
        ++launches;
        tstop();
        const size_t shm = gram_smem_floats(std::min(maxm, kGramSmem)) * 4;
        tonal_smem_limits(device);
        cudaMemsetAsync(flags, 0, 4, stream);
        tstart(kT_Gram);
        k_tonal_gram<<<nb, 256, shm, stream>>>(t_off, t_goff, t_echo, t_fac, flags, npx);
        ++launches;
        if (maxm > kGramSmem) {
            const size_t shb = gram_big_smem_bytes(maxm);
            k_tonal_gram_big<<<nb, 256, shb, stream>>>(t_off, t_goff, t_echo, t_fac, flags, npx);
            ++launches;
        }
        tstop();
        unsigned bad = 0;
        cudaMemcpyAsync(&bad, flags, 4, cudaMemcpyDeviceToHost, stream);
        if ((rc = sync("tonal local factors"))) return rc;
        if (bad) return fail(HDI_ERR_NONFINITE, "tonal: a local Gram matrix is not positive definite");
    }
    t_total = total;
    return sync("tonal setup");
}

void Ctx::tonal_residual(DFc y, DFc w) {
    const int parts = std::max(1, std::min(maxparts_, (mlist_n + 255) / 256));
    k_tonal_residual<<<dim3(parts, nch), 256, 0, stream>>>(arr(0), mview(0), cview(dfv[kF]), y, w, mlist, mlist_n,
                                                          tres, reducer(kSlotTonalR, parts),
                                                          reducer(kSlotTonalE, parts));
    ++launches;
}

// Raster-order list of the level-0 mask pixels (offsets y * pitch + x): the
// index set of the tonal residual, the Anderson vectors and the mask values.
int Ctx::mask_list() {
    int rc;
    std::vector<int> rc_h(H), rowoff(H + 1);
    if ((rc = lws.reserve(*this, std::max(lws.cap, (size_t)(H + 1) * 8 + 512), "mask list counts"))) return rc;
    int* drc = (int*)lws.take((size_t)(H + 1) * 4);
    k_row_counts<<<(H + 3) / 4, 128, 0, stream>>>(mview(0), drc);
    ++launches;
    cudaMemcpyAsync(rc_h.data(), drc, (size_t)H * 4, cudaMemcpyDeviceToHost, stream);
    if ((rc = sync("mask row counts"))) return rc;
    rowoff[0] = 0;
    for (int yy = 0; yy < H; ++yy) rowoff[yy + 1] = rowoff[yy] + rc_h[yy];
    const int M = rowoff[H];
    const size_t bytes = ((size_t)(H + 1) * 4 + 255) / 256 * 256 + ((size_t)std::max(M, 1) * 4 + 255) / 256 * 256;
    if ((rc = lws.reserve(*this, std::max(lws.cap, bytes), "mask list"))) return rc;
    int* drowoff = (int*)lws.take((size_t)(H + 1) * 4);
    mlist = (int*)lws.take((size_t)std::max(M, 1) * 4);
    mlist_n = M;
    cudaMemcpyAsync(drowoff, rowoff.data(), (size_t)(H + 1) * 4, cudaMemcpyHostToDevice, stream);
    k_compact_fill<<<(H + 3) / 4, 128, 0, stream>>>(mview(0), lev[0].P, drowoff, mlist);
    ++launches;
    return cuda_check(cudaGetLastError(), "mask list");
}

void Ctx::tonal_local(float* out) {
    const size_t shm = (size_t)4 * std::max(t_maxm, 1) * 4;   // at most 16 KB (m_i <= 1024)
    tstart(kT_Local);   // the nine colour launches as one timed unit
    for (int color = 0; color < 9; ++color) {
        LocalSolveArgs a;
        a.F = arr(0);
        a.nbx = t_nbx;
        a.nby = t_nby;
        a.stride = t_blk - kOv;
        a.blk = t_blk;
        a.lb = (t_blk == 64) ? 6 : 5;
        a.nch = nch;
        a.color = color;
        a.off = t_off;
        a.goff = t_goff;
        a.list = t_list;
        a.fac = t_fac;
        a.r = tres;
        a.out = out;
        const int hx = class_count(color % 3, t_nbx);
        const int hy = class_count(color / 3, t_nby);
        const long long blocks = (long long)hx * hy;
        if (blocks <= 0) continue;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)blocks);
        cfg.blockDim = dim3(32 * kLocalWarps);
        cfg.dynamicSmemBytes = shm;
        cfg.stream = stream;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = (p.pdl >= 0.5) ? 1 : 0;
        cudaLaunchKernelEx(&cfg, k_tonal_local, a);
        ++launches;
    }
    tstop();
}

// One wave of k_aa_gather<K>: its resident CTAs per SM (the K = 8 form holds
// 44 compensated sums per thread and runs one CTA per SM) times the SMs,
// shared among the channels, at most kAAParts per channel.
template <int K>
static void launch_aa_gather(AAArgs a, int new_slot, int device, cudaStream_t s) {
    static int occ = 0;
    if (occ == 0) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_aa_gather<K>, 256, 0) != cudaSuccess || v < 1) v = 1;
        occ = v;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1) sms = 1;
    a.nparts = std::max(1, std::min({kAAParts, sms * occ / a.nch, (a.M + 255) / 256}));
    k_aa_gather<K><<<dim3(a.nparts, a.nch), 256, 0, s>>>(a, new_slot);
}

// Solves the k x k least-squares normal equations of one channel by Cholesky
// in FP64, dropping the oldest columns while the matrix is numerically
// singular. A is packed as (r <= c) row by row, b follows.
static void aa_solve(const double* dots, int k, double* gam) {
    for (int j = 0; j < kAAMax; ++j) gam[j] = 0.0;
    double A[kAAMax][kAAMax], b[kAAMax];
    int q = 0;
    for (int r = 0; r < k; ++r)
        for (int c = r; c < k; ++c) { A[r][c] = A[c][r] = dots[q++]; }
    for (int r = 0; r < k; ++r) b[r] = dots[q++];
    for (int kk = k; kk >= 1; --kk) {
        double Lm[kAAMax][kAAMax];
        double dmax = 0.0;
        for (int r = 0; r < kk; ++r) dmax = std::max(dmax, A[r][r]);
        if (!(dmax > 0.0)) return;
        bool ok = true;
        for (int r = 0; r < kk && ok; ++r) {
            for (int c = 0; c <= r; ++c) {
                double s = A[r][c] + (r == c ? 1e-12 * dmax : 0.0);
                for (int j = 0; j < c; ++j) s -= Lm[r][j] * Lm[c][j];
                if (r == c) {
                    if (!(s > 1e-13 * dmax)) { ok = false; break; }
                    Lm[r][r] = std::sqrt(s);
                } else {
                    Lm[r][c] = s / Lm[c][c];
                }
            }
        }
        if (!ok) continue;
        double z[kAAMax];
        for (int r = 0; r < kk; ++r) {
            double s = b[r];
            for (int j = 0; j < r; ++j) s -= Lm[r][j] * z[j];
            z[r] = s / Lm[r][r];
        }
        for (int r = kk - 1; r >= 0; --r) {
            double s = z[r];
            for (int j = r + 1; j < kk; ++j) s -= Lm[j][r] * gam[j];
            gam[r] = s / Lm[r][r];
        }
        return;
    }
}

// One accelerated update g <- g + f_n - (dX + dF) gamma with f_n = P r_n in
// `fvfull` (iteration n of the outer loop).
int Ctx::tonal_aa_step(int n, const float* fvfull, DF G) {
    const int mwin = (int)p.tonal_anderson;
    const int ring = std::max(mwin, 1);
    const int k = std::min(mwin, n);
    AAArgs a;
    a.M = aa_M;
    a.cs = lev[0].cs;
    a.nch = nch;
    a.k = k;
    a.slot = n >= 1 ? (n - 1) % ring : 0;
    a.mwin = ring;
    a.beta = (float)p.tonal_anderson_beta;
    a.idx = aa_idx;
    a.fvfull = fvfull;
    a.fv = aa_fv;
    a.fvprev = aa_fvprev;
    a.dF = aa_dF;
    a.dX = aa_dX;
    a.g = G;
    a.gamma = aa_gam;
    a.partials = aa_part;
    a.out = aa_out;
    a.ticket = aa_ticket;
    a.nparts = std::max(1, std::min(kAAParts, (aa_M + 255) / 256));
    if (aa_M == 0) return HDI_OK;
    const int new_slot = (n >= 1 && mwin > 0) ? (n - 1) % ring : -1;
    tstart(kT_Anderson);
    ++launches;
    switch (k) {
        case 0: launch_aa_gather<0>(a, new_slot, device, stream); break;
        case 1: launch_aa_gather<1>(a, new_slot, device, stream); break;
        case 2: launch_aa_gather<2>(a, new_slot, device, stream); break;
        case 3: launch_aa_gather<3>(a, new_slot, device, stream); break;
        case 4: launch_aa_gather<4>(a, new_slot, device, stream); break;
        case 5: launch_aa_gather<5>(a, new_slot, device, stream); break;
        case 6: launch_aa_gather<6>(a, new_slot, device, stream); break;
        case 7: launch_aa_gather<7>(a, new_slot, device, stream); break;
        default: launch_aa_gather<8>(a, new_slot, device, stream); break;
    }
    tstop();
    if (k > 0) {
        const int nd = k * (k + 1) / 2 + k;
        double dots[4 * 64], gam[4 * kAAMax];
        cudaMemcpyAsync(dots, aa_out, (size_t)nch * nd * 8, cudaMemcpyDeviceToHost, stream);
        int rc = sync("Anderson dot products");
        if (rc) return rc;
        for (int c = 0; c < nch; ++c) aa_solve(dots + c * nd, k, gam + c * kAAMax);
        cudaMemcpyAsync(aa_gam, gam, (size_t)nch * kAAMax * 8, cudaMemcpyHostToDevice, stream);
    }
    const int blocks = std::max(1, std::min(1024, (aa_M + 255) / 256));
    tstart(kT_Anderson);
    k_aa_update<<<dim3(blocks, nch), 256, 0, stream>>>(a, mwin > 0 ? n % ring : 0);
    ++launches;
    tstop();
    return cuda_check(cudaGetLastError(), "Anderson update");
}

int Ctx::read_slot(int slot, double* out) {
    cudaMemcpyAsync(hscal, scal + slot * kMaxCh, (size_t)nch * 8, cudaMemcpyDeviceToHost, stream);
    int rc = sync("reading a reduction");
    if (rc) return rc;
    for (int c = 0; c < nch; ++c) out[c] = hscal[c];
    return HDI_OK;
}

int Ctx::tonal(const hdi_image* f, const hdi_mask* mask, const hdi_image* g0, hdi_image* g, double tol,
               hdi_stats* st) {
    int rc;
    if ((rc = cuda_check(cudaSetDevice(device), "cudaSetDevice"))) return rc;
    if ((rc = check_image(f, "f", -1, 0, 0))) return rc;
    if ((rc = check_image(g, "g", f->height, f->width, f->channels))) return rc;
    if (g->dtype != f->dtype) return fail(HDI_ERR_INVALID_ARG, "g: dtype differs from f");
    if (g0 && (rc = check_image(g0, "g0", f->height, f->width, f->channels))) return rc;
    if (!(tol > 0.0 && tol < 1.0)) return fail(HDI_ERR_INVALID_ARG, "tol must lie in (0, 1)");
    if ((rc = setup(f->height, f->width, f->channels))) return rc;
    long long ones = 0;
    if ((rc = load_mask(mask, &ones))) return rc;
    if (ones == 0) return fail(HDI_ERR_EMPTY_MASK, "empty mask: A is singular");
    const DFc F = cview(dfv[kF]);
    DF G = dfv[kG];
    f_lo_zero = true;
    const bool cgnr = p.tonal_method >= 0.5;
    const bool outer = p.tonal_max_iter >= 1;   // 0: only the initial values (e.g. the Voronoi initialisation)
    // the local factors depend on the mask only: a host f is copied to the
    // device on the side stream while their echo and Gram kernels run
    const bool overlap = f->location == HDI_HOST && !g0 && !cgnr && outer;
    struct PendingClear {   // the caller's f is not referenced past this call, on any return
        const hdi_image*& p;
        ~PendingClear() { p = nullptr; }
    } pending_clear{pending_upload};
    pending_upload = nullptr;
    if (overlap) {
        pending_upload = f;
    } else {
        if ((rc = load_image(f, dfv[kF]))) return rc;
        if (g0) {
            if ((rc = load_image(g0, G))) return rc;
        } else {
            cudaMemcpyAsync(G.hi, F.hi, (size_t)nch * lev[0].cs * 8, cudaMemcpyDeviceToDevice, stream);
        }
    }
    vcycles_run = 0;
    cudaMemsetAsync(counters + kCntLocal, 0, 16, stream);
    if ((rc = mask_list())) return rc;
    if (!cgnr && outer && (rc = tonal_setup())) return rc;
    if (overlap) {
        if (pending_upload) {   // the set-up did not reach its echo kernel: copy now
            pending_upload = nullptr;
            if ((rc = upload_begin(f))) return rc;
        }
        if ((rc = load_image(f, dfv[kF], nullptr, 0, true, true))) return rc;
        cudaMemcpyAsync(G.hi, F.hi, (size_t)nch * lev[0].cs * 8, cudaMemcpyDeviceToDevice, stream);
    }

    // the inner solves use their own local stop fraction (restored on exit)
    struct EtaSwap {
        Params& p;
        double keep, kpre, kpost;
        EtaSwap(Params& pp) : p(pp), keep(pp.oras_eta), kpre(pp.fine_pre), kpost(pp.fine_post) {
            p.oras_eta = p.tonal_oras_eta;
            p.fine_pre = p.tonal_fine_pre;
            p.fine_post = p.tonal_fine_post;
        }
        ~EtaSwap() {
            p.oras_eta = keep;
            p.fine_pre = kpre;
            p.fine_post = kpost;
        }
    } eta_swap(p);
    int vi_steps = 0;
    double vi_mse = 0.0;
    y_warm = false;
    if (p.tonal_init >= 0.5) {
        DF uk;
        if ((rc = tonal_vi(vi_steps, vi_mse, &uk))) return rc;
        if (uk.hi) {   // its inpainting warm-starts the first B g solve
            cudaMemcpyAsync(dfv[kY0].hi, uk.hi, (size_t)nch * lev[0].cs * 8, cudaMemcpyDeviceToDevice, stream);
            y_warm = true;
        }
    }
    const double ratio = p.tonal_inner_ratio;
    // ||B^T f||: w_f solves A w = (I - C) f.
    SolveSpec sw;
    sw.u[0] = dfv[kW0];
    sw.u[1] = dfv[kW1];
    sw.cur = 0;
    sw.rhs = RHS_SOURCE;
    sw.d = F;
    sw.y = DFc{nullptr, nullptr};
    sw.start = START_ZERO;
    sw.tol = 1e-3;   // ||B^T f|| only scales the stopping test; 0.1% is ample
    sw.max_iter = (int)p.max_vcycles;
    rc = solve(sw);
    if (rc != HDI_OK && rc != HDI_ERR_NOT_CONVERGED) return fail(rc, "tonal: B^T f solve: %s", err.c_str());
    tonal_residual(DFc{nullptr, nullptr}, cview(sw.u[sw.cur]));
    double btf2[kMaxCh], r2[kMaxCh], e2[kMaxCh];
    if ((rc = read_slot(kSlotTonalR, btf2))) return rc;
    int it = 0;
    double rel_max = 1.0, mse_last = 0.0;
    bool by_gain = false;
    if (cgnr) {
        if ((rc = tonal_cgnr(sw, btf2, tol, it, rel_max, mse_last, by_gain))) return rc;
    } else {
        SolveSpec sy;
        sy.u[0] = dfv[kY0];
        sy.u[1] = dfv[kY1];
        sy.cur = 0;
        sy.rhs = RHS_DATA;
        sy.d = cview(G);
        sy.start = y_warm ? START_WARM : START_FMG;
        sy.max_iter = (int)p.max_vcycles;
        sw.start = START_WARM;
        double rel_prev = 1.0, mse_prev = 0.0;
        const int max_it = (int)p.tonal_max_iter;
        // the MSE rule returns the best iterate seen (RAS is not monotone in the MSE)
        const DF Gbest = dfv[kU0];
        double mse_best = INFINITY, rel_best = 1.0;
        for (;; ++it) {
            const double tin = std::max(1e-13, std::min(p.tonal_inner_max, ratio * rel_prev));
            sy.tol = tin;
            rc = solve(sy);
            if (rc != HDI_OK && rc != HDI_ERR_NOT_CONVERGED)
                return fail(rc, "tonal: B g solve, iteration %d: %s", it, err.c_str());
            sy.start = START_WARM;
            sw.tol = tin;
            sw.y = cview(sy.u[sy.cur]);
            rc = solve(sw);
            if (rc != HDI_OK && rc != HDI_ERR_NOT_CONVERGED)
                return fail(rc, "tonal: adjoint solve, iteration %d: %s", it, err.c_str());
            tonal_residual(cview(sy.u[sy.cur]), cview(sw.u[sw.cur]));
            if ((rc = read_slot(kSlotTonalR, r2))) return rc;
            if ((rc = read_slot(kSlotTonalE, e2))) return rc;
            rel_max = 0.0;
            double esum = 0.0;
            for (int c = 0; c < nch; ++c) {
                if (!std::isfinite(r2[c])) return fail(HDI_ERR_NONFINITE, "tonal: non-finite residual");
                const double rel = btf2[c] > 0 ? std::sqrt(r2[c] / btf2[c]) : 0.0;
                rel_max = std::max(rel_max, rel);
                esum += e2[c] + sw.bnorm2[c];   // mask pixels + the rest (the adjoint right-hand side)
            }
            mse_last = esum / ((double)nch * H * W);
            if (p.trace > 0)
                fprintf(stderr, "[hdi tonal] it %d rel %.3e mse %.6f inner tol %.2e y: %d vc rel %.2e  w: %d vc rel %.2e\n",
                        it, rel_max, mse_last, tin, sy.iterations, sy.rel_max, sw.iterations, sw.rel_max);
            if (rel_max <= tol || it >= max_it) break;
            if (p.tonal_mse_gain > 0 && it > 0 && mse_prev - mse_last < p.tonal_mse_gain * mse_prev) {
                by_gain = true;
                if (mse_best < mse_last) {
                    cudaMemcpyAsync(G.hi, Gbest.hi, (size_t)nch * lev[0].cs * 8, cudaMemcpyDeviceToDevice, stream);
                    mse_last = mse_best;
                    rel_max = rel_best;
                }
                break;
            }
            if (p.tonal_mse_gain > 0 && mse_last < mse_best) {
                cudaMemcpyAsync(Gbest.hi, G.hi, (size_t)nch * lev[0].cs * 8, cudaMemcpyDeviceToDevice, stream);
                mse_best = mse_last;
                rel_best = rel_max;
            }
            rel_prev = rel_max;
            mse_prev = mse_last;
            float* fvfull = lev[0].xb;   // free between solves
            cudaMemsetAsync(fvfull, 0, (size_t)nch * lev[0].cs * 4, stream);
            tonal_local(fvfull);
            if ((rc = tonal_aa_step(it, fvfull, G))) return rc;
        }
    }
    if ((rc = store_image(cview(G), g, true))) return rc;
    if (st) {
        unsigned long long li[2] = {0, 0};
        cudaMemcpy(li, counters + kCntLocal, 16, cudaMemcpyDeviceToHost);
        st->iterations = it;
        st->vcycles = vcycles_run;
        st->local_iters = (int64_t)li[0];
        st->rel_res = rel_max;
        // without outer iterations the initialisation's own MSE (inpaintings
        // at vi_inner_tol) is the better figure than the first evaluation's
        st->mse = (!outer && p.tonal_init >= 0.5) ? vi_mse : mse_last;
        st->init_steps = vi_steps;
    }
    if ((rc = tflush())) return rc;
    if (rel_max > tol && !by_gain && outer)
        return fail(HDI_ERR_NOT_CONVERGED, "tonal: relative residual %.3e after %d %s iterations", rel_max, it,
                    cgnr ? "CGNR" : "RAS");
    return HDI_OK;
}

// CGNR outer loop (Sec. 5.1, "Improvements"; kernels in cgnr.cuh). On entry
// G holds g0 and sw the warm adjoint solve of B^T f. Per iteration: w = B p
// (inpainting of p from full multigrid), the alpha step on y and g, then
// y = B g re-solved warm from the updated y (so that inexact inner solves do
// not accumulate in the residual), z = B^T (f - y) and the new direction.
// Inner tolerances follow the RAS driver: ratio * current relative residual,
// at most tonal_inner_max.
int Ctx::tonal_cgnr(SolveSpec& sw, const double* btf2, double tol, int& it, double& rel_max, double& mse_last,
                    bool& by_gain) {
    int rc;
    const DF G = dfv[kG];
    const DF P = dfv[kP];
    const double ratio = p.tonal_inner_ratio;
    const int max_it = (int)p.tonal_max_iter;
    const int parts = std::min(maxparts_, 4 * 148);
    const dim3 vgrid(parts, nch);
    const MaskView m0 = mview(0);
    SolveSpec sy;   // y = B g
    sy.u[0] = dfv[kY0];
    sy.u[1] = dfv[kY1];
    sy.cur = 0;
    sy.rhs = RHS_DATA;
    sy.d = cview(G);
    sy.start = y_warm ? START_WARM : START_FMG;
    sy.max_iter = (int)p.max_vcycles;
    SolveSpec spw;  // w = B p
    spw.u[0] = dfv[kU0];
    spw.u[1] = dfv[kU1];
    spw.rhs = RHS_DATA;
    spw.d = cview(P);
    spw.max_iter = (int)p.max_vcycles;
    double r2[kMaxCh], e2[kMaxCh];
    double mse_prev = 0.0;
    sw.start = START_WARM;
    // z = B^T (f - y) and the figures of the current iterate
    auto evaluate = [&](double tin) -> int {
        int r;
        sy.tol = tin;
        r = solve(sy);
        if (r != HDI_OK && r != HDI_ERR_NOT_CONVERGED) return fail(r, "CGNR: B g solve: %s", err.c_str());
        sy.start = START_WARM;
        sw.tol = tin;
        sw.y = cview(sy.u[sy.cur]);
        r = solve(sw);
        if (r != HDI_OK && r != HDI_ERR_NOT_CONVERGED) return fail(r, "CGNR: adjoint solve: %s", err.c_str());
        tonal_residual(cview(sy.u[sy.cur]), cview(sw.u[sw.cur]));
        if ((r = read_slot(kSlotTonalR, r2))) return r;
        if ((r = read_slot(kSlotTonalE, e2))) return r;
        rel_max = 0.0;
        double esum = 0.0;
        for (int c = 0; c < nch; ++c) {
            if (!std::isfinite(r2[c])) return fail(HDI_ERR_NONFINITE, "CGNR: non-finite residual");
            rel_max = std::max(rel_max, btf2[c] > 0 ? std::sqrt(r2[c] / btf2[c]) : 0.0);
            esum += e2[c] + sw.bnorm2[c];   // mask pixels + the rest (the adjoint right-hand side)
        }
        mse_last = esum / ((double)nch * H * W);
        return HDI_OK;
    };
    if ((rc = evaluate(std::max(1e-13, std::min(p.tonal_inner_max, ratio))))) return rc;
    k_cgnr_direction<<<vgrid, kCgnrThreads, 0, stream>>>(arr(0), m0, tres, P, scal + kSlotTonalR * kMaxCh,
                                                           scal + kSlotCgZ * kMaxCh, 1);
    ++launches;
    for (it = 0;; ++it) {
        if (p.trace > 0)
            fprintf(stderr, "[hdi cgnr] it %d rel %.3e mse %.6f  y: %d vc  w: %d vc\n", it, rel_max, mse_last,
                    sy.iterations, sw.iterations);
        if (rel_max <= tol || it >= max_it) break;
        if (p.tonal_mse_gain > 0 && it > 0 && mse_prev - mse_last < p.tonal_mse_gain * mse_prev) {
            by_gain = true;
            break;
        }
        const double tin = std::max(1e-13, std::min(p.tonal_inner_max, ratio * rel_max));
        mse_prev = mse_last;
        // w = B p
        spw.cur = 0;
        spw.start = START_FMG;
        spw.tol = tin;
        rc = solve(spw);
        if (rc != HDI_OK && rc != HDI_ERR_NOT_CONVERGED) return fail(rc, "CGNR: B p solve: %s", err.c_str());
        const DF w = spw.u[spw.cur];
        k_cgnr_dots<<<vgrid, kCgnrThreads, 0, stream>>>(arr(0), m0, cview(w), tres, cview(P), reducer(kSlotCgW, parts),
                                                         reducer(kSlotCgZP, parts));
        // y += alpha w (the warm start of the next B g solve), g += alpha p
        k_cgnr_step<<<vgrid, kCgnrThreads, 0, stream>>>(arr(0), m0, sy.u[sy.cur], cview(w), G, cview(P),
                                                         scal + kSlotTonalR * kMaxCh, scal + kSlotCgZP * kMaxCh,
                                                         scal + kSlotCgW * kMaxCh, scal + kSlotCgZ * kMaxCh);
        launches += 2;
        if ((rc = evaluate(tin))) return rc;
        k_cgnr_direction<<<vgrid, kCgnrThreads, 0, stream>>>(arr(0), m0, tres, P, scal + kSlotTonalR * kMaxCh,
                                                               scal + kSlotCgZ * kMaxCh, 0);
        ++launches;
    }
    return cuda_check(cudaGetLastError(), "CGNR");
}

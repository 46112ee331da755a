// stencil.cuh -- streaming stencil kernels of the multigrid cycle
// (Sec. 3.2): mask packing and restriction, residual + restriction,
// prolongation + correction, the FP64 residual of the refinement loop, and
// staging between caller images and the internal FP64 layout.
//
// Transfers (cell-centred, Sec. 3.2 / Sec. 3.3):
//   mask  : a coarse pixel is known if any of its (up to) four children is;
//   data  : a coarse known pixel holds the mean of its known children;
//   r     : coarse right-hand side = sum of the children's residuals
//           (= 4 x their mean; the coarse operator is the plain stencil,
//           i.e. L_H = L / 4 for H = 2h) and 0 on coarse known pixels,
//           where the coarse error is pinned to zero;
//   P     : bilinear interpolation between coarse cell centres (weights
//           9/16, 3/16, 3/16, 1/16), constant extension at the border.
#pragma once
#include "common.cuh"

// ---------------------------------------------------------------- masks ---

// uint8 0/1 mask (any row stride) -> bit-packed level-0 mask; counts the
// ones and flags values other than 0/1.
__global__ void k_pack_mask(const uint8_t* __restrict__ m, long long rs, int H, int W,
                            uint32_t* __restrict__ bits, int wpitch,
                            unsigned long long* count, unsigned* bad) {
    const int wx = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (y >= H || wx >= wpitch) return;
    uint32_t word = 0;
    int ones = 0;
    const int x0 = wx * 32;
    for (int i = 0; i < 32; ++i) {
        const int x = x0 + i;
        if (x < W) {
            const uint8_t v = m[(size_t)y * rs + x];
            if (v > 1) atomicOr(bad, 1u);
            if (v) { word |= 1u << i; ++ones; }
        }
    }
    bits[(size_t)y * wpitch + wx] = word;
    if (ones) atomicAdd(count, (unsigned long long)ones);
}

// Bit-packed mask -> uint8 0/1 (caller layout).
__global__ void k_unpack_mask(const uint32_t* __restrict__ bits, int wpitch, int H, int W,
                              uint8_t* __restrict__ m, long long rs) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W || y >= H) return;
    m[(size_t)y * rs + x] = (bits[(size_t)y * wpitch + (x >> 5)] >> (x & 31)) & 1u;
}

// Compress the even bits of a 64-bit word into 32 bits.
__device__ __forceinline__ uint32_t even_bits(uint64_t x) {
    x &= 0x5555555555555555ull;
    x = (x | (x >> 1)) & 0x3333333333333333ull;
    x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
    x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
    x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
    return (uint32_t)x;
}

// Coarse mask bit = OR of the 2x2 children (Sec. 3.3).
__global__ void k_restrict_mask(MaskView f, uint32_t* __restrict__ cbits, int cH, int cW, int cwp) {
    const int wx = blockIdx.x * blockDim.x + threadIdx.x;
    const int Y = blockIdx.y;
    if (Y >= cH || wx >= cwp) return;
    uint32_t out = 0;
    if (wx * 32 < cW) {
        const int fw = 2 * wx;   // fine words 2wx, 2wx+1 hold this word's children
        uint64_t r = 0;
        for (int fy = 2 * Y; fy <= 2 * Y + 1 && fy < f.H; ++fy) {
            const uint32_t* row = f.bits + (size_t)fy * f.wpitch;
            const uint64_t lo = (fw < f.wpitch) ? row[fw] : 0u;
            const uint64_t hi = (fw + 1 < f.wpitch) ? row[fw + 1] : 0u;
            r |= lo | (hi << 32);
        }
        out = even_bits(r | (r >> 1));
        const int valid = cW - wx * 32;
        if (valid < 32) out &= (1u << valid) - 1u;
    }
    cbits[(size_t)Y * cwp + wx] = out;
}

// --------------------------------------------------------- level arrays ---

struct LevelArr {
    int H, W, pitch;   // pitch in elements
    long long cs;      // elements per channel
};

// FMG data pyramid: coarse known pixel = mean of its known children, else 0.
__global__ void k_restrict_data(LevelArr F, MaskView fm, const float* __restrict__ fb,
                                LevelArr C, float* __restrict__ cb) {
    const int X = blockIdx.x * blockDim.x + threadIdx.x;
    const int Y = blockIdx.y * blockDim.y + threadIdx.y;
    const int ch = blockIdx.z;
    if (X >= C.W || Y >= C.H) return;
    float s = 0.f;
    int n = 0;
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
            const int x = 2 * X + dx, y = 2 * Y + dy;
            if (x < F.W && y < F.H && fm.known(x, y)) {
                s += fb[ch * F.cs + (size_t)y * F.pitch + x];
                ++n;
            }
        }
    cb[ch * C.cs + (size_t)Y * C.pitch + X] = n ? s / (float)n : 0.f;
}

// Fine residual r = b - A x on unknown pixels (difference form), 0 on known.
__device__ __forceinline__ float fine_residual(const float* __restrict__ x, const float* __restrict__ b,
                                               const LevelArr& F, const MaskView& m, int px, int py) {
    if (m.known(px, py)) return 0.f;
    const size_t i = (size_t)py * F.pitch + px;
    const float xc = x[i];
    float lap = 0.f;
    if (px > 0) lap += xc - x[i - 1];
    if (px + 1 < F.W) lap += xc - x[i + 1];
    if (py > 0) lap += xc - x[i - F.pitch];
    if (py + 1 < F.H) lap += xc - x[i + F.pitch];
    return b[i] - lap;
}

// Coarse right-hand side b_H = sum of the children's residuals (0 on coarse
// known pixels) and ||b_H||^2 per channel. Block 32x8 over coarse pixels;
// each CTA walks TILE_ROWS consecutive 8-row bands so that few CTAs take
// part in the grid reduction.
#define TILE_ROWS 16
__global__ void __launch_bounds__(256) k_restrict_residual(LevelArr F, MaskView fm, const float* __restrict__ x,
                                                           const float* __restrict__ b, LevelArr C, MaskView cm,
                                                           float* __restrict__ cb, GridReduce red) {
    const int X = blockIdx.x * blockDim.x + threadIdx.x;
    const int ch = blockIdx.z;
    const float* xc = x + ch * F.cs;
    const float* bc = b + ch * F.cs;
    float sq = 0.f;
    for (int band = 0; band < TILE_ROWS; ++band) {
        const int Y = (blockIdx.y * TILE_ROWS + band) * blockDim.y + threadIdx.y;
        if (X < C.W && Y < C.H) {
            float s = 0.f;
            if (!cm.known(X, Y)) {
                for (int dy = 0; dy < 2; ++dy)
                    for (int dx = 0; dx < 2; ++dx) {
                        const int px = 2 * X + dx, py = 2 * Y + dy;
                        if (px < F.W && py < F.H) s += fine_residual(xc, bc, F, fm, px, py);
                    }
            }
            cb[ch * C.cs + (size_t)Y * C.pitch + X] = s;
            sq += s * s;
        }
    }
    const double tot = (double)block_sum_f(sq);
    grid_reduce_commit(red, ch, blockIdx.y * gridDim.x + blockIdx.x, tot);
}

// Bilinear cell-centred prolongation of coarse e at fine pixel (px, py).
__device__ __forceinline__ float prolong_at(const float* __restrict__ e, const LevelArr& C, int px, int py) {
    const int X = px >> 1, Y = py >> 1;
    const int Xn = (px & 1) ? min(X + 1, C.W - 1) : max(X - 1, 0);
    const int Yn = (py & 1) ? min(Y + 1, C.H - 1) : max(Y - 1, 0);
    const float* r0 = e + (size_t)Y * C.pitch;
    const float* r1 = e + (size_t)Yn * C.pitch;
    return 0.5625f * r0[X] + 0.1875f * (r0[Xn] + r1[X]) + 0.0625f * r1[Xn];
}

// Tiles of 32x8 pixels with a one-pixel halo in shared memory.
#define PT_W 32
#define PT_H 8

// MODE 0 (V-cycle): xout = xin + P e on unknown pixels, xin on known ones;
// MODE 1 (FMG):     xout = b on known pixels, P e on unknown ones;
// MODE 2 (start):   xout = b on known pixels, 0 on unknown ones (e unused).
// Then ||b - A xout||^2 per channel (the next sweep's local stop rule).
template <int MODE>
__global__ void __launch_bounds__(PT_W * PT_H) k_prolong(LevelArr F, MaskView fm, const float* __restrict__ xin,
                                                         const float* __restrict__ b, float* __restrict__ xout,
                                                         LevelArr C, const float* __restrict__ e, GridReduce red) {
    __shared__ float t[PT_H + 2][PT_W + 2];
    const int ch = blockIdx.z;
    const int bx0 = blockIdx.x * PT_W;
    const float* xc = (MODE == 0) ? xin + ch * F.cs : nullptr;
    const float* bc = b + ch * F.cs;
    const float* ec = (MODE == 2) ? nullptr : e + ch * C.cs;
    float sq = 0.f;
    for (int band = 0; band < TILE_ROWS; ++band) {
        const int by0 = (blockIdx.y * TILE_ROWS + band) * PT_H;
        if (by0 >= F.H) break;
        __syncthreads();
        for (int i = threadIdx.y * PT_W + threadIdx.x; i < (PT_W + 2) * (PT_H + 2); i += PT_W * PT_H) {
            const int ty = i / (PT_W + 2), tx = i - ty * (PT_W + 2);
            const int px = min(max(bx0 + tx - 1, 0), F.W - 1);
            const int py = min(max(by0 + ty - 1, 0), F.H - 1);
            const size_t idx = (size_t)py * F.pitch + px;
            float v;
            if (fm.known(px, py)) v = (MODE == 0) ? xc[idx] : bc[idx];
            else if (MODE == 2) v = 0.f;
            else v = (MODE == 0 ? xc[idx] : 0.f) + prolong_at(ec, C, px, py);
            t[ty][tx] = v;
        }
        __syncthreads();
        const int px = bx0 + threadIdx.x, py = by0 + threadIdx.y;
        if (px < F.W && py < F.H) {
            const int tx = threadIdx.x + 1, ty = threadIdx.y + 1;
            const float v = t[ty][tx];
            xout[ch * F.cs + (size_t)py * F.pitch + px] = v;
            if (!fm.known(px, py)) {
                float lap = 0.f;
                if (px > 0) lap += v - t[ty][tx - 1];
                if (px + 1 < F.W) lap += v - t[ty][tx + 1];
                if (py > 0) lap += v - t[ty - 1][tx];
                if (py + 1 < F.H) lap += v - t[ty + 1][tx];
                const float r = bc[(size_t)py * F.pitch + px] - lap;
                sq += r * r;
            }
        }
    }
    const double tot = (double)block_sum_f(sq);
    grid_reduce_commit(red, ch, blockIdx.y * gridDim.x + blockIdx.x, tot);
}

// ------------------------------------------- double-float refinement step ---
//
// The level-0 iterate, the data and the tonal vectors are held as
// double-float pairs (hi, lo) of FP32 numbers with value hi + lo and
// |lo| <= ulp(hi)/2, about 48 significant bits. The refinement residual is
// formed with error-free transformations (Knuth's TwoSum, Dekker's
// Fast2Sum), so it is as accurate as an FP64 evaluation while every
// operation runs on the FP32 pipes (the FP64 rate of the target is a small
// fraction of its FP32 rate).

struct DF {
    float* hi;      // [nch][H][pitch]
    float* lo;      // same layout, second half of the allocation
};
struct DFc {
    const float* hi;
    const float* lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    e = b - (s - a);
}
// (ah, al) + (bh, bl), renormalised.
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& sh, float& sl) {
    float s, e;
    two_sum(ah, bh, s, e);
    e += al + bl;
    fast_two_sum(s, e, sh, sl);
}
// Split of an FP64 value into a double-float pair.
__device__ __forceinline__ void df_from_d(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

// Right-hand side of the fine-level system:
//   RHS_DATA   : b = C d            (d = f for inpainting, d = g for B g)
//   RHS_SOURCE : b = (I - C)(d - y) (the adjoint solve of Sec. 5.1)
enum { RHS_DATA = 0, RHS_SOURCE = 1 };
// Value of the iterate on unknown pixels before the residual:
//   INIT_KEEP   : u = uin
//   INIT_UPDATE : u = uin + e (FP32 correction from the V-cycle)
//   INIT_FROM32 : u = x (FP32 FMG result)
//   INIT_ZERO   : u = 0
// In every mode known pixels take their Dirichlet value (d, or 0 for
// RHS_SOURCE), so u_K is exact. The result goes to uout, which must not alias
// uin (neighbouring tiles read uin as their halo).
enum { INIT_KEEP = 0, INIT_UPDATE = 1, INIT_FROM32 = 2, INIT_ZERO = 3 };

struct ResArgs {
    LevelArr F;           // level-0 geometry
    MaskView m;
    DFc uin;              // iterate before the step
    DF uout;              // iterate after the step
    const float* x32;     // INIT_UPDATE: correction e; INIT_FROM32: x
    DFc d;                // data (RHS_DATA) or minuend (RHS_SOURCE)
    DFc y;                // subtrahend (RHS_SOURCE; hi == nullptr means 0)
    float* r32;           // out: residual rounded to FP32 (V-cycle right-hand side)
    GridReduce red_r;     // ||r||^2 per channel
    GridReduce red_b;     // ||b||^2 per channel (only if want_b)
    int want_b;
};

template <int RHS, int INIT>
__global__ void __launch_bounds__(PT_W * PT_H) k_residual_df(ResArgs a) {
    __shared__ float th[PT_H + 2][PT_W + 2];
    __shared__ float tl[PT_H + 2][PT_W + 2];
    const int ch = blockIdx.z;
    const int bx0 = blockIdx.x * PT_W;
    const long long co = ch * a.F.cs;
    float rr = 0.f, bb2 = 0.f;
    for (int band = 0; band < TILE_ROWS; ++band) {
    const int by0 = (blockIdx.y * TILE_ROWS + band) * PT_H;
    if (by0 >= a.F.H) break;
    __syncthreads();
    for (int i = threadIdx.y * PT_W + threadIdx.x; i < (PT_W + 2) * (PT_H + 2); i += PT_W * PT_H) {
        const int ty = i / (PT_W + 2), tx = i - ty * (PT_W + 2);
        const int px = min(max(bx0 + tx - 1, 0), a.F.W - 1);
        const int py = min(max(by0 + ty - 1, 0), a.F.H - 1);
        const size_t idx = co + (size_t)py * a.F.pitch + px;
        float h, l;
        if (a.m.known(px, py)) {
            if (RHS == RHS_DATA) { h = a.d.hi[idx]; l = a.d.lo[idx]; }
            else { h = 0.f; l = 0.f; }
        } else if (INIT == INIT_KEEP) {
            h = a.uin.hi[idx]; l = a.uin.lo[idx];
        } else if (INIT == INIT_UPDATE) {
            df_add(a.uin.hi[idx], a.uin.lo[idx], a.x32[idx], 0.f, h, l);
        } else if (INIT == INIT_FROM32) {
            h = a.x32[idx]; l = 0.f;
        } else {
            h = 0.f; l = 0.f;
        }
        th[ty][tx] = h;
        tl[ty][tx] = l;
    }
    __syncthreads();
    const int px = bx0 + threadIdx.x, py = by0 + threadIdx.y;
    if (px < a.F.W && py < a.F.H) {
        const int tx = threadIdx.x + 1, ty = threadIdx.y + 1;
        const size_t idx = co + (size_t)py * a.F.pitch + px;
        const float ch_ = th[ty][tx], cl = tl[ty][tx];
        a.uout.hi[idx] = ch_;
        a.uout.lo[idx] = cl;
        float r = 0.f;
        if (a.m.known(px, py)) {
            if (RHS == RHS_DATA) { const float bh = a.d.hi[idx] + a.d.lo[idx]; bb2 += bh * bh; }
        } else {
            // lap = sum over in-image neighbours of (u_c - u_n), error-free:
            // the hi differences are summed with TwoSum, every rounding error
            // and the lo differences go to the low-order accumulator.
            float sh = 0.f, sl = 0.f;
            const int nx[4] = {tx - 1, tx + 1, tx, tx};
            const int ny[4] = {ty, ty, ty - 1, ty + 1};
            const bool ok[4] = {px > 0, px + 1 < a.F.W, py > 0, py + 1 < a.F.H};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (ok[k]) {
                    float dh, dl, s2, e2;
                    two_sum(ch_, -th[ny[k]][nx[k]], dh, dl);
                    dl += cl - tl[ny[k]][nx[k]];
                    two_sum(sh, dh, s2, e2);
                    sh = s2;
                    sl += e2 + dl;
                }
            }
            float bh = 0.f, bl = 0.f;
            if (RHS == RHS_SOURCE) {
                const float yh = a.y.hi ? a.y.hi[idx] : 0.f, yl = a.y.hi ? a.y.lo[idx] : 0.f;
                df_add(a.d.hi[idx], a.d.lo[idx], -yh, -yl, bh, bl);
                bb2 += bh * bh;
            }
            float rh, rl;
            df_add(bh, bl, -sh, -sl, rh, rl);
            r = rh + rl;
        }
        a.r32[idx] = r;
        rr += r * r;
    }
    }
    const double tot = (double)block_sum_f(rr);
    grid_reduce_commit(a.red_r, ch, blockIdx.y * gridDim.x + blockIdx.x, tot);
    if (a.want_b) {
        const double totb = (double)block_sum_f(bb2);
        grid_reduce_commit(a.red_b, ch, blockIdx.y * gridDim.x + blockIdx.x, totb);
    }
}

// ------------------------------------------------------------ staging ---

// Caller image (F32/F64, any strides) -> internal double-float pair;
// flags non-finite values. For FP64 input, lo2 (if given) receives the bits
// below the pair, (v - hi) - lo, which are exact in FP32, so that
// hi + lo + lo2 reproduces v exactly.
template <typename T>
__global__ void k_load_image(const T* __restrict__ src, long long rs, long long cs, LevelArr F, DF dst,
                             float* __restrict__ lo2, unsigned* bad) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int ch = blockIdx.z;
    if (x >= F.W) return;
    const T v = src[ch * cs + (size_t)y * rs + x];
    if (!isfinite(v)) atomicOr(bad, 1u);
    float h, l;
    if (sizeof(T) == 8) df_from_d((double)v, h, l);
    else { h = (float)v; l = 0.f; }
    const size_t idx = ch * F.cs + (size_t)y * F.pitch + x;
    dst.hi[idx] = h;
    dst.lo[idx] = l;
    if (lo2) lo2[idx] = (sizeof(T) == 8) ? (float)(((double)v - (double)h) - (double)l) : 0.f;
}

// Internal double-float -> caller image; with zero_off_mask, pixels off the
// mask are 0. known_lo2 (if given) adds the third component of the data on
// known pixels, so inpainted FP64 output equals f there bit for bit.
template <typename T>
__global__ void k_store_image(DFc src, LevelArr F, MaskView m, int zero_off_mask, const float* __restrict__ known_lo2,
                              T* __restrict__ dst, long long rs, long long cs) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int ch = blockIdx.z;
    if (x >= F.W) return;
    const size_t idx = ch * F.cs + (size_t)y * F.pitch + x;
    T v;
    if (sizeof(T) == 8) {
        double dv = (double)src.hi[idx] + (double)src.lo[idx];
        if (known_lo2 && m.known(x, y)) dv += (double)known_lo2[idx];
        v = (T)dv;
    } else {
        v = (T)(src.hi[idx] + src.lo[idx]);
    }
    if (zero_off_mask && !m.known(x, y)) v = (T)0;
    dst[ch * cs + (size_t)y * rs + x] = v;
}

// Data at known pixels -> FP32 (FMG right-hand side on level 0), 0 elsewhere.
__global__ void k_data_to_f32(DFc d, LevelArr F, MaskView m, float* __restrict__ out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int ch = blockIdx.z;
    if (x >= F.W) return;
    const size_t idx = ch * F.cs + (size_t)y * F.pitch + x;
    out[idx] = m.known(x, y) ? d.hi[idx] + d.lo[idx] : 0.f;
}

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
// known pixels) and ||b_H||^2 per channel. Block 32x8 over coarse pixels.
__global__ void __launch_bounds__(256) k_restrict_residual(LevelArr F, MaskView fm, const float* __restrict__ x,
                                                           const float* __restrict__ b, LevelArr C, MaskView cm,
                                                           float* __restrict__ cb, GridReduce red) {
    const int X = blockIdx.x * blockDim.x + threadIdx.x;
    const int Y = blockIdx.y * blockDim.y + threadIdx.y;
    const int ch = blockIdx.z;
    const float* xc = x + ch * F.cs;
    const float* bc = b + ch * F.cs;
    double sq = 0.0;
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
        sq = (double)s * (double)s;
    }
    const double tot = block_sum_d(sq);
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
    const int bx0 = blockIdx.x * PT_W, by0 = blockIdx.y * PT_H;
    const float* xc = (MODE == 0) ? xin + ch * F.cs : nullptr;
    const float* bc = b + ch * F.cs;
    const float* ec = (MODE == 2) ? nullptr : e + ch * C.cs;
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
    double sq = 0.0;
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
            sq = (double)r * (double)r;
        }
    }
    const double tot = block_sum_d(sq);
    grid_reduce_commit(red, ch, blockIdx.y * gridDim.x + blockIdx.x, tot);
}

// ------------------------------------------------- FP64 refinement step ---

// Right-hand side of the fine-level system in FP64:
//   RHS_DATA   : b = C d            (d = f for inpainting, d = g for B g)
//   RHS_SOURCE : b = (I - C)(d - y) (the adjoint solve of Sec. 5.1)
enum { RHS_DATA = 0, RHS_SOURCE = 1 };
// Value of the FP64 iterate on unknown pixels before the residual:
//   INIT_KEEP   : u = uin
//   INIT_UPDATE : u = uin + e (FP32 correction from the V-cycle)
//   INIT_FROM32 : u = x (FP32 FMG result)
//   INIT_ZERO   : u = 0
// In every mode known pixels take their Dirichlet value (d, or 0 for
// RHS_SOURCE), so u_K is exact in FP64. The result goes to uout, which must
// not alias uin (neighbouring tiles read uin as their halo).
enum { INIT_KEEP = 0, INIT_UPDATE = 1, INIT_FROM32 = 2, INIT_ZERO = 3 };

struct Res64Args {
    LevelArr F;           // level-0 geometry
    MaskView m;
    const double* uin;    // FP64 iterate before the step
    double* uout;         // FP64 iterate after the step
    const float* x32;     // INIT_UPDATE: correction e; INIT_FROM32: x
    const double* d;      // data (RHS_DATA) or minuend (RHS_SOURCE)
    const double* y;      // subtrahend (RHS_SOURCE; nullptr = 0)
    float* r32;           // out: residual in FP32 (V-cycle right-hand side)
    GridReduce red_r;     // ||r||^2 per channel
    GridReduce red_b;     // ||b||^2 per channel (only if want_b)
    int want_b;
};

template <int RHS, int INIT>
__global__ void __launch_bounds__(PT_W * PT_H) k_residual64(Res64Args a) {
    __shared__ double t[PT_H + 2][PT_W + 2];
    const int ch = blockIdx.z;
    const int bx0 = blockIdx.x * PT_W, by0 = blockIdx.y * PT_H;
    const long long co = ch * a.F.cs;
    for (int i = threadIdx.y * PT_W + threadIdx.x; i < (PT_W + 2) * (PT_H + 2); i += PT_W * PT_H) {
        const int ty = i / (PT_W + 2), tx = i - ty * (PT_W + 2);
        const int px = min(max(bx0 + tx - 1, 0), a.F.W - 1);
        const int py = min(max(by0 + ty - 1, 0), a.F.H - 1);
        const size_t idx = co + (size_t)py * a.F.pitch + px;
        double v;
        if (a.m.known(px, py)) {
            v = (RHS == RHS_DATA) ? a.d[idx] : 0.0;
        } else {
            if (INIT == INIT_KEEP) v = a.uin[idx];
            else if (INIT == INIT_UPDATE) v = a.uin[idx] + (double)a.x32[idx];
            else if (INIT == INIT_FROM32) v = (double)a.x32[idx];
            else v = 0.0;
        }
        t[ty][tx] = v;
    }
    __syncthreads();
    const int px = bx0 + threadIdx.x, py = by0 + threadIdx.y;
    double sq = 0.0, sb = 0.0;
    if (px < a.F.W && py < a.F.H) {
        const int tx = threadIdx.x + 1, ty = threadIdx.y + 1;
        const size_t idx = co + (size_t)py * a.F.pitch + px;
        const double v = t[ty][tx];
        a.uout[idx] = v;
        double r, bv;
        if (a.m.known(px, py)) {
            bv = (RHS == RHS_DATA) ? a.d[idx] : 0.0;
            r = bv - v;
        } else {
            bv = (RHS == RHS_DATA) ? 0.0 : (a.d[idx] - (a.y ? a.y[idx] : 0.0));
            double lap = 0.0;
            if (px > 0) lap += v - t[ty][tx - 1];
            if (px + 1 < a.F.W) lap += v - t[ty][tx + 1];
            if (py > 0) lap += v - t[ty - 1][tx];
            if (py + 1 < a.F.H) lap += v - t[ty + 1][tx];
            r = bv - lap;
        }
        a.r32[idx] = (float)r;
        sq = r * r;
        sb = bv * bv;
    }
    const double tot = block_sum_d(sq);
    grid_reduce_commit(a.red_r, ch, blockIdx.y * gridDim.x + blockIdx.x, tot);
    if (a.want_b) {
        const double totb = block_sum_d(sb);
        grid_reduce_commit(a.red_b, ch, blockIdx.y * gridDim.x + blockIdx.x, totb);
    }
}

// ------------------------------------------------------------ staging ---

// Caller image (F32/F64, any strides) -> internal FP64 [nch][H][pitch];
// flags non-finite values.
template <typename T>
__global__ void k_load_image(const T* __restrict__ src, long long rs, long long cs, LevelArr F,
                             double* __restrict__ dst, unsigned* bad) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int ch = blockIdx.z;
    if (x >= F.W) return;
    const double v = (double)src[ch * cs + (size_t)y * rs + x];
    if (!isfinite(v)) atomicOr(bad, 1u);
    dst[ch * F.cs + (size_t)y * F.pitch + x] = v;
}

// Internal FP64 -> caller image; with zero_off_mask, pixels off the mask are 0.
template <typename T>
__global__ void k_store_image(const double* __restrict__ src, LevelArr F, MaskView m, int zero_off_mask,
                              T* __restrict__ dst, long long rs, long long cs) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int ch = blockIdx.z;
    if (x >= F.W) return;
    double v = src[ch * F.cs + (size_t)y * F.pitch + x];
    if (zero_off_mask && !m.known(x, y)) v = 0.0;
    dst[ch * cs + (size_t)y * rs + x] = (T)v;
}

// FP64 data at known pixels -> FP32 (FMG right-hand side on level 0), 0 elsewhere.
__global__ void k_data_to_f32(const double* __restrict__ d, LevelArr F, MaskView m, float* __restrict__ out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int ch = blockIdx.z;
    if (x >= F.W) return;
    const size_t idx = ch * F.cs + (size_t)y * F.pitch + x;
    out[idx] = m.known(x, y) ? (float)d[idx] : 0.f;
}

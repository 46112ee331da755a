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
#include <type_traits>
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

// Coarse mask bit = OR of the 2x2 children (Sec. 3.3). `known` (may be
// null) accumulates the coarse level's known pixels over all planes.
__global__ void k_restrict_mask(MaskView f, uint32_t* __restrict__ cbits, int cH, int cW, int cwp,
                                unsigned long long* known) {
    const int wx = blockIdx.x * blockDim.x + threadIdx.x;
    const int Y = blockIdx.y;
    const bool valid = Y < cH && wx < cwp;
    f.bits += (size_t)blockIdx.z * f.cstride;           // mask plane
    cbits += (size_t)blockIdx.z * (size_t)cH * cwp;
    uint32_t out = 0;
    if (valid && wx * 32 < cW) {
        const int fw = 2 * wx;   // fine words 2wx, 2wx+1 hold this word's children
        uint64_t r = 0;
        for (int fy = 2 * Y; fy <= 2 * Y + 1 && fy < f.H; ++fy) {
            const uint32_t* row = f.bits + (size_t)fy * f.wpitch;
            const uint64_t lo = (fw < f.wpitch) ? row[fw] : 0u;
            const uint64_t hi = (fw + 1 < f.wpitch) ? row[fw + 1] : 0u;
            r |= lo | (hi << 32);
        }
        out = even_bits(r | (r >> 1));
        const int nvalid = cW - wx * 32;
        if (nvalid < 32) out &= (1u << nvalid) - 1u;
    }
    if (valid) cbits[(size_t)Y * cwp + wx] = out;
    if (known) {
        const unsigned n = __reduce_add_sync(HDI_FULL, (unsigned)__popc(out));
        if ((threadIdx.x & 31) == 0 && n) atomicAdd(known, (unsigned long long)n);
    }
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
    fm = fm.ch(ch);
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
// known pixels) and ||b_H||^2 per channel. Column strips over the fine grid
// (see CS_ROWS below): each lane forms the fine residual of its column, two
// consecutive rows are summed in registers and lane pairs (2j, 2j+1) are
// combined by a shuffle.
#define CS_ROWS 64
#define CS_CHUNK 4
#ifndef RES_CHUNK
#define RES_CHUNK 1
#endif

// Rows per CTA of the column-strip kernels: long strips on large levels (few
// CTAs take part in each grid reduction), short ones on small levels, where
// the serial walk down the rows would otherwise dominate. Always even (the
// restriction pairs rows) and, from CS_CHUNK rows on, a multiple of it.
static inline int strip_rows(int H, int W, int nch) {
    const long long cols = (long long)((W + 127) / 128) * nch;
    long long rows = (long long)H * cols / 2400;   // aim at >= ~2400 CTAs
    rows = (rows < 4 ? 4LL : (rows > CS_ROWS ? (long long)CS_ROWS : rows));
    if (rows >= CS_CHUNK) return (int)((rows + CS_CHUNK - 1) / CS_CHUNK * CS_CHUNK);
    return (int)(rows + (rows & 1));
}

// The column-strip kernels walk their rows in chunks of CS_CHUNK: every load
// of a chunk (the rows below, the halo columns of lanes 0 and 31, mask words,
// right-hand sides) is issued before any of its arithmetic, so a warp keeps
// a chunk's worth of independent loads in flight instead of one row's.
// Loads past the strip's last row are clamped into the image and unused.

// Halo column of a strip's edge lanes: lane 0 reads column x0 - 1, lane 31
// column x0 + 32 (the neighbouring strips' edge columns), when inside.
struct StripHalo {
    bool on;
    int col;
};
__device__ __forceinline__ StripHalo strip_halo(int lane, int px, int pxc, int W) {
    StripHalo h;
    h.on = (lane == 0 && px > 0) || (lane == 31 && px + 1 < W);
    h.col = h.on ? ((lane == 0) ? px - 1 : px + 1) : pxc;
    return h;
}

// ---- quad strips ----
// A warp covers 128 columns of `rows` rows: lane l holds columns x0 + 4l ..
// x0 + 4l + 3 as one float4 (16-byte loads: rows are 128-byte aligned and x0
// is a multiple of 128), so one load instruction moves 512 bytes. A CTA
// stacks four warps on consecutive row blocks of one strip. Lanes 0 and 31
// read the neighbouring strips' edge columns; lanes past the image still
// take part in the shuffles with clamped loads. Rows are walked in chunks of
// QS_CHUNK, every load of a chunk issued before its arithmetic. The kernels
// keep one chunk buffer and run at 64-72 registers (7-8 CTAs per SM): more
// resident warps hide the load latency better than a second register buffer
// with the next chunk's loads in flight (measured faster on the 4K RGB
// workload). On level 0 the next chunk can instead be staged in shared
// memory (cp.async, no registers; stage_loads), which the residual and the
// restriction gain from.
#define QS_COLS 128
#define QS_CHUNK 2

// Rows per warp: the same number of warps as column strips of
// strip_rows(H, W, nch) rows would give, at least one chunk, even.
static inline int quad_rows(int H, int W, int nch) {
    int r = strip_rows(H, W, nch) / 4;
    r = (r + QS_CHUNK - 1) / QS_CHUNK * QS_CHUNK;
    return r < QS_CHUNK ? QS_CHUNK : r;
}
static inline dim3 quad_grid(int H, int W, int nch, int rows) {
    return dim3((W + QS_COLS - 1) / QS_COLS, (H + 4 * rows - 1) / (4 * rows), nch);
}

struct QuadLane {
    int lane, x0, c0, cq;    // strip origin, first column of the lane, clamped load column
    bool act[4];             // column c0 + j inside the image
    bool lin[4], rin[4];     // left / right neighbour of column c0 + j inside the image
    bool hon;                // lane 0 / 31 reads a halo column
    int hcol;                // that column (clamped when unused)
    int shift;               // bit of column c0 in its mask word
    int mword;               // index of that word within a mask row
};
__device__ __forceinline__ QuadLane quad_lane(int x0, const LevelArr& F, const MaskView& m) {
    QuadLane q;
    q.lane = threadIdx.x & 31;
    q.x0 = x0;
    q.c0 = x0 + 4 * q.lane;
    q.cq = min(q.c0, F.pitch - 4);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        q.act[j] = q.c0 + j < F.W;
        q.lin[j] = q.c0 + j > 0;
        q.rin[j] = q.c0 + j + 1 < F.W;
    }
    q.hon = (q.lane == 0 && x0 > 0) || (q.lane == 31 && x0 + QS_COLS < F.W);
    q.hcol = q.hon ? ((q.lane == 0) ? x0 - 1 : x0 + QS_COLS) : min(q.c0, F.W - 1);
    q.shift = q.c0 & 31;
    q.mword = min(q.c0 >> 5, m.wpitch - 1);
    return q;
}
__device__ __forceinline__ void f4_to(const float4 v, float (&a)[4]) {
    a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
}
// b - A x at the lane's four columns of one row (difference form; absent
// neighbours contribute nothing), given the rows above / below and the halo.
__device__ __forceinline__ void quad_residual(const QuadLane& q, const float (&c)[4], const float (&u)[4],
                                             const float (&d)[4], const float (&bv)[4], float hv, bool hasu,
                                             bool hasd, float (&r)[4]) {
    float lw = __shfl_up_sync(HDI_FULL, c[3], 1);
    float rw = __shfl_down_sync(HDI_FULL, c[0], 1);
    if (q.lane == 0) lw = hv;
    if (q.lane == 31) rw = hv;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float l = (j == 0) ? lw : c[j - 1];
        const float rr = (j == 3) ? rw : c[j + 1];
        float lap = 0.f;
        if (q.lin[j]) lap += c[j] - l;
        if (q.rin[j]) lap += c[j] - rr;
        if (hasu) lap += c[j] - u[j];
        if (hasd) lap += c[j] - d[j];
        r[j] = bv[j] - lap;
    }
}

// quad_residual for a lane whose four columns, their left and right
// neighbours and the rows above and below all lie inside the image.
__device__ __forceinline__ void quad_residual_interior(int lane, const float (&c)[4], const float (&u)[4],
                                                      const float (&d)[4], const float (&bv)[4], float hv,
                                                      float (&r)[4]) {
    float lw = __shfl_up_sync(HDI_FULL, c[3], 1);
    float rw = __shfl_down_sync(HDI_FULL, c[0], 1);
    if (lane == 0) lw = hv;
    if (lane == 31) rw = hv;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float l = (j == 0) ? lw : c[j - 1];
        const float rr = (j == 3) ? rw : c[j + 1];
        r[j] = bv[j] - (((c[j] - l) + (c[j] - rr)) + ((c[j] - u[j]) + (c[j] - d[j])));
    }
}

// Read access to one field of a chunk staged in shared memory, with the
// interface of the register chunk's arrays: element k sits k * 128 words
// further (the [field][thread] layout of 128-thread CTAs); a field that was
// not staged reads as zero.
struct StagedF4 {
    const float4* p;
    bool on;
    __device__ __forceinline__ float4 operator[](int k) const {
        return on ? p[k * 128] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
};
struct StagedU32 {
    const uint32_t* p;
    bool on;
    __device__ __forceinline__ uint32_t operator[](int k) const { return on ? p[k * 128] : 0u; }
};
struct StagedF32 {
    const uint32_t* p;
    bool on;
    __device__ __forceinline__ float operator[](int k) const { return on ? __uint_as_float(p[k * 128]) : 0.f; }
};
// Staging layout of the restriction (dynamic shared memory, [slot][field]
// [thread] as the residual kernel's): float4 fields x of rows yb+1, yb+2 and
// b of rows yb, yb+1; word fields the halo's x of rows yb, yb+1, the mask
// words of rows yb, yb+1 and the coarse mask word of row yb/2. Two slots
// (one chunk in flight ahead) keep 7 CTAs per SM.
struct RStage {
    static constexpr int NV = 2 * QS_CHUNK, NW = 2 * QS_CHUNK + 1, NSLOT = 2;
    static constexpr size_t bytes = (size_t)NSLOT * 128 * (NV * 16 + NW * 4);
};
struct StagedRestrict {
    StagedF4 Xd, Bv;
    StagedF32 Hv;
    StagedU32 Mw;
    uint32_t Cw;
};

// r = b - A x on level F with 2x2 sums into the coarse right-hand side
// (restriction, Sec. 3.2), zero on coarse known pixels, and ||r_c||^2 per
// channel. Quad strips: the lane's four columns feed two coarse columns.
// Warps whose strip and row block (with the rows above and below) lie inside
// the image run a variant without border tests or clamped rows (IN).
// Body shared by the plain launch (one level, all channels of one image) and
// the batched launch (StripTask table); returns the thread's share of
// ||r_c||^2 for the caller's block and grid reduction.
__device__ __forceinline__ float restrict_residual_body(LevelArr F, MaskView fm, const float* __restrict__ x,
                                                        const float* __restrict__ b, LevelArr C, MaskView cm,
                                                        float* __restrict__ cb, int rows, int bx, int by, int ch) {
    constexpr int CR = QS_CHUNK;
    static_assert(CR == 2, "one coarse row per chunk");
    pdl_trigger();
    fm = fm.ch(ch);
    cm = cm.ch(ch);
    const int y0 = (by * 4 + (threadIdx.x >> 5)) * rows;
    const int y1 = min(y0 + rows, F.H);
    const int x0 = bx * QS_COLS;
    const QuadLane q = quad_lane(x0, F, fm);
    const bool interior = x0 > 0 && x0 + QS_COLS < F.W && y0 > 0 && y0 + rows + 1 <= F.H;
    pdl_wait();
    const float* xc = x + ch * F.cs;
    const float* bc = b + ch * F.cs;
    float sq = 0.f;
    extern __shared__ float4 qs_dyn[];
    const bool staged = dyn_smem_bytes() >= RStage::bytes;
    auto sv = [&](int sl, int f) { return qs_dyn + ((size_t)(sl * RStage::NV + f) * 128 + threadIdx.x); };
    auto sw = [&](int sl, int f) {
        return reinterpret_cast<uint32_t*>(qs_dyn + (size_t)RStage::NSLOT * RStage::NV * 128) +
               ((size_t)(sl * RStage::NW + f) * 128 + threadIdx.x);
    };
    auto body = [&](auto in_tag) {
        constexpr bool IN = decltype(in_tag)::value;
        const uint32_t* mrow = fm.bits + q.mword;
        const int X = q.c0 >> 1;                  // first of the lane's two coarse columns
        const uint32_t* cmw = cm.bits + min(X >> 5, cm.wpitch - 1);
        auto rowc = [&](int y) { return IN ? y : min(y, F.H - 1); };
        float up[4] = {0.f, 0.f, 0.f, 0.f}, cen[4];
        if (IN || y0 > 0) f4_to(*reinterpret_cast<const float4*>(xc + (size_t)(y0 - 1) * F.pitch + q.cq), up);
        f4_to(*reinterpret_cast<const float4*>(xc + (size_t)y0 * F.pitch + q.cq), cen);
        float pair[2] = {0.f, 0.f};
        struct Chunk {
            float4 Xd[CR], Bv[CR];
            float Hv[CR];
            uint32_t Mw[CR], Cw;
        };
        auto load = [&](Chunk& c, int yb) {
#pragma unroll
            for (int k = 0; k < CR; ++k) {
                const size_t ry = (size_t)rowc(yb + k) * F.pitch;
                c.Xd[k] = *reinterpret_cast<const float4*>(xc + (size_t)rowc(yb + k + 1) * F.pitch + q.cq);
                c.Bv[k] = *reinterpret_cast<const float4*>(bc + ry + q.cq);
                c.Hv[k] = q.hon ? xc[ry + q.hcol] : 0.f;
                c.Mw[k] = mrow[(size_t)rowc(yb + k) * fm.wpitch];
            }
            c.Cw = cmw[(size_t)(IN ? (yb >> 1) : min(yb >> 1, C.H - 1)) * cm.wpitch];   // one coarse row
        };
        // c: a Chunk in registers, or a StagedRestrict view of the staging slots
        auto compute = [&](const auto& c, int yb) {
#pragma unroll
            for (int k = 0; k < CR; ++k) {
                const int y = yb + k;
                if (!IN && y >= y1) break;
                float dn[4], bv[4], r[4];
                f4_to(c.Xd[k], dn);
                f4_to(c.Bv[k], bv);
                if (IN) {
                    quad_residual_interior(q.lane, cen, up, dn, bv, c.Hv[k], r);
                } else {
                    quad_residual(q, cen, up, dn, bv, c.Hv[k], y > 0, y + 1 < F.H, r);
                }
                const uint32_t nib = c.Mw[k] >> q.shift;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const bool unk = (IN || q.act[j]) && !((nib >> j) & 1u);
                    pair[j >> 1] += unk ? r[j] : 0.f;
                }
                if ((y & 1) || (!IN && y + 1 == F.H)) {
                    const int Y = y >> 1;
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        const bool ok = IN || (q.act[2 * t] && X + t < C.W);
                        const float v = ((c.Cw >> ((X & 31) + t)) & 1u) ? 0.f : pair[t];
                        if (ok) {
                            cb[ch * C.cs + (size_t)Y * C.pitch + X + t] = v;
                            sq += v * v;
                        }
                        pair[t] = 0.f;
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    up[j] = cen[j];
                    cen[j] = dn[j];
                }
            }
        };
        if (staged) {
            // copies of chunk yb into slot sl, from the addresses load() reads
            auto stage = [&](int sl, int yb) {
#pragma unroll
                for (int k = 0; k < CR; ++k) {
                    const size_t ry = (size_t)rowc(yb + k) * F.pitch;
                    cpa16(sv(sl, k), xc + (size_t)rowc(yb + k + 1) * F.pitch + q.cq);
                    cpa16(sv(sl, CR + k), bc + ry + q.cq);
                    if (q.hon) cpa4(sw(sl, k), xc + ry + q.hcol);
                    cpa4(sw(sl, CR + k), mrow + (size_t)rowc(yb + k) * fm.wpitch);
                }
                cpa4(sw(sl, 2 * CR), cmw + (size_t)(IN ? (yb >> 1) : min(yb >> 1, C.H - 1)) * cm.wpitch);
            };
            auto view = [&](int sl) {
                StagedRestrict c;
                c.Xd = {sv(sl, 0), true};
                c.Bv = {sv(sl, CR), true};
                c.Hv = {sw(sl, 0), q.hon};
                c.Mw = {sw(sl, CR), true};
                c.Cw = *sw(sl, 2 * CR);
                return c;
            };
            // two slots in rotation: the next chunk in flight while one is computed
            stage(0, y0);
            cpa_commit();
            int sl = 0;
            for (int yb = y0; yb < y1; yb += CR) {
                if (yb + CR < y1) stage(sl ^ 1, yb + CR);
                cpa_commit();
                cpa_wait<1>();   // chunk yb has landed
                compute(view(sl), yb);
                sl ^= 1;
            }
        } else {
            for (int yb = y0; yb < y1; yb += CR) {
                Chunk A;
                load(A, yb);
                compute(A, yb);
            }
        }
    };
    if (interior) body(std::true_type{});
    else if (y0 < F.H) body(std::false_type{});
    return sq;
}

__global__ void __launch_bounds__(128, 7) k_restrict_residual(LevelArr F, MaskView fm, const float* __restrict__ x,
                                                           const float* __restrict__ b, LevelArr C, MaskView cm,
                                                           float* __restrict__ cb, GridReduce red, int rows) {
    const float sq = restrict_residual_body(F, fm, x, b, C, cm, cb, rows, blockIdx.x, blockIdx.y, blockIdx.z);
    const double tot = (double)block_sum_f(sq);
    grid_reduce_commit(red, blockIdx.z, blockIdx.y * gridDim.x + blockIdx.x, tot);
}

// One (image, channel) of a batched launch of the quad-strip kernels:
// geometry, mask planes and buffers of that channel (pointers at the
// channel's plane, so the bodies run with ch = 0) and its grid.
struct StripTask {
    LevelArr F, C;          // level and its coarse level
    MaskView fm, cm;        // mask planes (chmask = nullptr)
    const float* x;         // iterate (restriction; prolongation MODE 0)
    const float* b;         // right-hand side on F
    float* xout;            // prolongation output
    const float* e;         // coarse correction (prolongation MODE 0/1)
    float* cb;              // restriction output (right-hand side on C)
    int rows;               // rows per warp
    int gx, gy;             // strips and row blocks of this task
};

__global__ void __launch_bounds__(128, 7) k_restrict_residual_b(const StripTask* __restrict__ tasks,
                                                             const int* __restrict__ cta0, int ntasks, SegReduce red) {
    const int t = find_task(cta0, ntasks, blockIdx.x);
    const StripTask tk = tasks[t];
    const int local = blockIdx.x - cta0[t];
    const float sq = restrict_residual_body(tk.F, tk.fm, tk.x, tk.b, tk.C, tk.cm, tk.cb, tk.rows, local % tk.gx,
                                            local / tk.gx, 0);
    const double tot = (double)block_sum_f(sq);
    seg_reduce_commit(red, t, local, tot);
}

// ||b - A x||^2 per channel on one level (quad strips, FP32).
__global__ void __launch_bounds__(128, 8) k_level_residual_norm(LevelArr F, MaskView fm, const float* __restrict__ x,
                                                             const float* __restrict__ b, GridReduce red, int rows) {
    constexpr int CR = QS_CHUNK;
    pdl_trigger();
    const int ch = blockIdx.z;
    fm = fm.ch(ch);
    const int y0 = (blockIdx.y * 4 + (threadIdx.x >> 5)) * rows;
    const int y1 = min(y0 + rows, F.H);
    const int x0 = blockIdx.x * QS_COLS;
    const QuadLane q = quad_lane(x0, F, fm);
    const bool interior = x0 > 0 && x0 + QS_COLS < F.W && y0 > 0 && y0 + rows + 1 <= F.H;
    pdl_wait();
    const float* xc = x + ch * F.cs;
    const float* bc = b + ch * F.cs;
    float sq = 0.f;
    auto body = [&](auto in_tag) {
        constexpr bool IN = decltype(in_tag)::value;   // no border tests, no clamped rows
        auto rowc = [&](int y) { return IN ? y : min(y, F.H - 1); };
        const uint32_t* mrow = fm.bits + q.mword;
        float up[4] = {0.f, 0.f, 0.f, 0.f}, cen[4];
        if (IN || y0 > 0) f4_to(*reinterpret_cast<const float4*>(xc + (size_t)(y0 - 1) * F.pitch + q.cq), up);
        f4_to(*reinterpret_cast<const float4*>(xc + (size_t)y0 * F.pitch + q.cq), cen);
        struct Chunk {
            float4 Xd[CR], Bv[CR];
            float Hv[CR];
            uint32_t Mw[CR];
        };
        auto load = [&](Chunk& c, int yb) {
#pragma unroll
            for (int k = 0; k < CR; ++k) {
                const size_t ry = (size_t)rowc(yb + k) * F.pitch;
                c.Xd[k] = *reinterpret_cast<const float4*>(xc + (size_t)rowc(yb + k + 1) * F.pitch + q.cq);
                c.Bv[k] = *reinterpret_cast<const float4*>(bc + ry + q.cq);
                c.Hv[k] = q.hon ? xc[ry + q.hcol] : 0.f;
                c.Mw[k] = mrow[(size_t)rowc(yb + k) * fm.wpitch];
            }
        };
        auto compute = [&](const Chunk& c, int yb) {
#pragma unroll
            for (int k = 0; k < CR; ++k) {
                const int y = yb + k;
                if (!IN && y >= y1) break;
                float dn[4], bv[4], r[4];
                f4_to(c.Xd[k], dn);
                f4_to(c.Bv[k], bv);
                if (IN) quad_residual_interior(q.lane, cen, up, dn, bv, c.Hv[k], r);
                else quad_residual(q, cen, up, dn, bv, c.Hv[k], y > 0, y + 1 < F.H, r);
                const uint32_t nib = c.Mw[k] >> q.shift;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const bool unk = (IN || q.act[j]) && !((nib >> j) & 1u);
                    if (unk) sq += r[j] * r[j];
                    up[j] = cen[j];
                    cen[j] = dn[j];
                }
            }
        };
        for (int yb = y0; yb < y1; yb += CR) {
            Chunk A;
            load(A, yb);
            compute(A, yb);
        }
    };
    if (interior) body(std::true_type{});
    else if (y0 < F.H) body(std::false_type{});
    const double tot = (double)block_sum_f(sq);
    grid_reduce_commit(red, ch, blockIdx.y * gridDim.x + blockIdx.x, tot);
}

// MODE 0 (V-cycle): xout = xin + P e on unknown pixels, xin on known ones;
// MODE 1 (FMG):     xout = b on known pixels, P e on unknown ones;
// MODE 2 (start):   xout = b on known pixels, 0 on unknown ones (e unused).
// P is bilinear cell-centred interpolation (Sec. 3.2): fine pixel (x, y) takes
// 3/4 of its coarse cell (X, Y) = (x/2, y/2) and 1/4 of the neighbouring
// coarse cell on its side in each direction, applied as a horizontal pass on
// the coarse rows h(R) = 3/4 e[R][X] + 1/4 e[R][Xn] and a vertical one,
// 3/4 h(Y) + 1/4 h(Yn) (clamped at the border).
// Then ||b - A xout||^2 per channel (the next sweep's local stop rule).
// Quad strips: the lane's four fine columns lie over two coarse cells
// (X0, X0 + 1), read as one float2; the outer neighbours X0 - 1 and X0 + 2
// come from the adjacent lanes by shuffles (edge lanes load them), and they
// are also the halo columns' cells, so lanes 0 and 31 interpolate the halo
// column without further coarse loads. Each coarse row is interpolated once
// and reused by the fine rows above and below it.
template <int MODE>
__device__ __forceinline__ float prolong_body(LevelArr F, MaskView fm, const float* __restrict__ xin,
                                              const float* __restrict__ b, float* __restrict__ xout, LevelArr C,
                                              const float* __restrict__ e, int rows, int bx, int by, int ch) {
    constexpr int CR = QS_CHUNK;
    constexpr int NS = CR / 2 + 2;   // coarse rows per chunk: (yb/2 - 1) .. (yb/2 + CR/2)
    pdl_trigger();
    fm = fm.ch(ch);
    const int y0 = (by * 4 + (threadIdx.x >> 5)) * rows;
    const int y1 = min(y0 + rows, F.H);
    const QuadLane q = quad_lane(bx * QS_COLS, F, fm);
    pdl_wait();
    const int lane = q.lane;
    const float* xc = (MODE == 0) ? xin + ch * F.cs : nullptr;
    const float* bc = b + ch * F.cs;
    const float* ec = (MODE == 2) ? nullptr : e + ch * C.cs;
    float* xo = xout + ch * F.cs;
    float sq = 0.f;
    if (y0 < F.H) {
        const uint32_t* mrow = fm.bits + q.mword;
        const uint32_t* hrow = fm.bits + (q.hcol >> 5);
        const int hbit = q.hcol & 31;
        const int X0 = q.c0 >> 1;
        const int Xq = min(X0, C.pitch - 2);          // float2 load column (clamped for idle lanes)
        const bool in1 = X0 + 1 < C.W, in2 = X0 + 2 < C.W, inm = X0 > 0;
        // the neighbour cells of the edge lanes: X0 - 1 (lane 0), X0 + 2 (lane 31)
        const int Xe = (lane == 0) ? max(X0 - 1, 0) : min(X0 + 2, C.W - 1);
        // horizontal interpolation of coarse row R at the lane's four columns
        // (h[0..3]) and at its halo column (hh, lanes 0 / 31)
        auto hinterp = [&](float2 ev, float ee, float (&h)[4], float& hh) {
            const float e0 = ev.x;
            const float e1 = in1 ? ev.y : ev.x;
            float em = __shfl_up_sync(HDI_FULL, e1, 1);
            float e2 = __shfl_down_sync(HDI_FULL, e0, 1);
            if (lane == 0) em = ee;
            if (lane == 31) e2 = ee;
            if (!inm) em = e0;
            if (!in2) e2 = e1;
            h[0] = __fadd_rn(__fmul_rn(0.75f, e0), __fmul_rn(0.25f, em));
            h[1] = __fadd_rn(__fmul_rn(0.75f, e0), __fmul_rn(0.25f, e1));
            h[2] = __fadd_rn(__fmul_rn(0.75f, e1), __fmul_rn(0.25f, e0));
            h[3] = __fadd_rn(__fmul_rn(0.75f, e1), __fmul_rn(0.25f, e2));
            hh = (lane == 0) ? __fadd_rn(__fmul_rn(0.75f, em), __fmul_rn(0.25f, e0))
                             : __fadd_rn(__fmul_rn(0.75f, e2), __fmul_rn(0.25f, e1));
        };
        auto cload = [&](int R, float2& ev, float& ee) {
            if (MODE == 2) { ev = make_float2(0.f, 0.f); ee = 0.f; return; }
            const float* row = ec + (size_t)min(max(R, 0), C.H - 1) * C.pitch;
            ev = *reinterpret_cast<const float2*>(row + Xq);
            ee = (lane == 0 || lane == 31) ? row[Xe] : 0.f;
        };
        auto fval = [&](bool known, float xv, float bv, float hY, float hYn) -> float {
            if (known) return (MODE == 0) ? xv : bv;
            if (MODE == 2) return 0.f;
            const float pe = __fadd_rn(__fmul_rn(0.75f, hY), __fmul_rn(0.25f, hYn));
            return (MODE == 0 ? xv : 0.f) + pe;
        };
        // coarse slots: S[j] / SH[j] = interpolated coarse row cb + j (clamped)
        float S[NS][4], SH[NS];
        {
            const int cb0 = (y0 >> 1) - 1;
            float2 ev;
            float ee;
            cload(cb0, ev, ee);
            hinterp(ev, ee, S[0], SH[0]);
            cload(cb0 + 1, ev, ee);
            hinterp(ev, ee, S[1], SH[1]);
        }
        // window: up = xout(y0 - 1) (Y slot 0, Yn slot 1), cen = xout(y0) (Y slot 1, Yn slot 0)
        float up[4] = {0.f, 0.f, 0.f, 0.f}, cen[4];
        {
            float xv[4] = {0.f, 0.f, 0.f, 0.f}, bv[4];
            const size_t r0 = (size_t)y0 * F.pitch + q.cq;
            if (MODE == 0) f4_to(*reinterpret_cast<const float4*>(xc + r0), xv);
            f4_to(*reinterpret_cast<const float4*>(bc + r0), bv);
            const uint32_t w0 = mrow[(size_t)y0 * fm.wpitch];
#pragma unroll
            for (int j = 0; j < 4; ++j) cen[j] = fval((w0 >> (q.shift + j)) & 1u, xv[j], bv[j], S[1][j], S[0][j]);
            if (y0 > 0) {
                const size_t rm = (size_t)(y0 - 1) * F.pitch + q.cq;
                if (MODE == 0) f4_to(*reinterpret_cast<const float4*>(xc + rm), xv);
                f4_to(*reinterpret_cast<const float4*>(bc + rm), bv);
                const uint32_t wm = mrow[(size_t)(y0 - 1) * fm.wpitch];
#pragma unroll
                for (int j = 0; j < 4; ++j) up[j] = fval((wm >> (q.shift + j)) & 1u, xv[j], bv[j], S[0][j], S[1][j]);
            }
        }
        struct Chunk {
            float4 Xd[CR], Bd[CR + 1];
            uint32_t Mw[CR + 1], Hm[CR];
            float Hx[CR], Hb[CR];
            float2 Ev[NS - 2];
            float Ee[NS - 2];
        };
        auto load = [&](Chunk& c, int yb) {
            const int cb = (yb >> 1) - 1;
#pragma unroll
            for (int j = 0; j < NS - 2; ++j) cload(cb + 2 + j, c.Ev[j], c.Ee[j]);
#pragma unroll
            for (int k = 0; k <= CR; ++k) {
                const int y = min(yb + k, F.H - 1);
                c.Bd[k] = *reinterpret_cast<const float4*>(bc + (size_t)y * F.pitch + q.cq);
                c.Mw[k] = mrow[(size_t)y * fm.wpitch];
            }
#pragma unroll
            for (int k = 0; k < CR; ++k) {
                const int y = min(yb + k, F.H - 1);
                const size_t ry = (size_t)y * F.pitch;
                if (MODE == 0)
                    c.Xd[k] = *reinterpret_cast<const float4*>(xc + (size_t)min(yb + k + 1, F.H - 1) * F.pitch + q.cq);
                else
                    c.Xd[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                c.Hx[k] = (MODE == 0 && q.hon) ? xc[ry + q.hcol] : 0.f;
                c.Hb[k] = q.hon ? bc[ry + q.hcol] : 0.f;
                c.Hm[k] = q.hon ? hrow[(size_t)y * fm.wpitch] : 0u;
            }
        };
        auto compute = [&](const Chunk& c, int yb) {
#pragma unroll
            for (int j = 0; j < NS - 2; ++j) hinterp(c.Ev[j], c.Ee[j], S[2 + j], SH[2 + j]);
#pragma unroll
            for (int k = 0; k < CR; ++k) {
                const int y = yb + k;
                if (y >= y1) break;
                // row y + 1 (k + 1 relative): Y slot ((k+1) >> 1) + 1, Yn on its side
                const int kd = k + 1;
                const int sY = (kd >> 1) + 1, sYn = (kd & 1) ? sY + 1 : sY - 1;
                float dn[4] = {0.f, 0.f, 0.f, 0.f};
                if (y + 1 < F.H) {
                    float xv[4], bv[4];
                    f4_to(c.Xd[k], xv);
                    f4_to(c.Bd[k + 1], bv);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        dn[j] = fval((c.Mw[k + 1] >> (q.shift + j)) & 1u, xv[j], bv[j], S[sY][j], S[sYn][j]);
                }
                const int hY = (k >> 1) + 1, hYn = (k & 1) ? hY + 1 : hY - 1;
                const float hv = fval((c.Hm[k] >> hbit) & 1u, c.Hx[k], c.Hb[k], SH[hY], SH[hYn]);
                float bv[4], r[4];
                f4_to(c.Bd[k], bv);
                quad_residual(q, cen, up, dn, bv, hv, y > 0, y + 1 < F.H, r);
                float* orow = xo + (size_t)y * F.pitch + q.c0;
                if (q.act[3]) {
                    *reinterpret_cast<float4*>(orow) = make_float4(cen[0], cen[1], cen[2], cen[3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (q.act[j]) orow[j] = cen[j];
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const bool unk = q.act[j] && !((c.Mw[k] >> (q.shift + j)) & 1u);
                    if (unk) sq += r[j] * r[j];
                    up[j] = cen[j];
                    cen[j] = dn[j];
                }
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
#pragma unroll
                for (int t = 0; t < 4; ++t) S[j][t] = S[NS - 2 + j][t];
                SH[j] = SH[NS - 2 + j];
            }
        };
        for (int yb = y0; yb < y1; yb += CR) {
            Chunk A;
            load(A, yb);
            compute(A, yb);
        }
    }
    return sq;
}

template <int MODE>
__global__ void __launch_bounds__(128, 7) k_prolong(LevelArr F, MaskView fm, const float* __restrict__ xin,
                                                 const float* __restrict__ b, float* __restrict__ xout,
                                                 LevelArr C, const float* __restrict__ e, GridReduce red, int rows) {
    const float sq = prolong_body<MODE>(F, fm, xin, b, xout, C, e, rows, blockIdx.x, blockIdx.y, blockIdx.z);
    const double tot = (double)block_sum_f(sq);
    grid_reduce_commit(red, blockIdx.z, blockIdx.y * gridDim.x + blockIdx.x, tot);
}

template <int MODE>
__global__ void __launch_bounds__(128, 7) k_prolong_b(const StripTask* __restrict__ tasks, const int* __restrict__ cta0,
                                                   int ntasks, SegReduce red) {
    const int t = find_task(cta0, ntasks, blockIdx.x);
    const StripTask tk = tasks[t];
    const int local = blockIdx.x - cta0[t];
    const float sq = prolong_body<MODE>(tk.F, tk.fm, tk.x, tk.b, tk.xout, tk.C, tk.e, tk.rows, local % tk.gx,
                                        local / tk.gx, 0);
    const double tot = (double)block_sum_f(sq);
    seg_reduce_commit(red, t, local, tot);
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
// RHS_SOURCE), so u_K is exact. INIT_KEEP works in place (uout = uin) and
// stores only the known pixels: every reader takes a known pixel's value
// from d, never from u, so no tile depends on the order of those stores.
// The other modes write every pixel to uout, which must not alias uin
// (neighbouring tiles read uin as their halo).
enum { INIT_KEEP = 0, INIT_UPDATE = 1, INIT_FROM32 = 2, INIT_ZERO = 3 };

// The residual kernel's chunk fields as views of its staging slots.
struct StagedRows {
    StagedF4 Uh, Ul, E, Dh, Dl, Yh, Yl, KDh, KDl;
    StagedU32 Mw, Hm;
    StagedF32 HUh, HUl, HE, HDh, HDl;
};

struct ResArgs {
    LevelArr F;           // level-0 geometry
    MaskView m;
    DFc uin;              // iterate before the step
    DF uout;              // iterate after the step
    const float* x32;     // INIT_UPDATE: correction e; INIT_FROM32: x
    DFc d;                // data (RHS_DATA) or minuend (RHS_SOURCE)
    DFc y;                // subtrahend (RHS_SOURCE; hi == nullptr means 0)
    float* r32;           // out: residual rounded to FP32 (V-cycle right-hand side)
    int rows;             // rows per CTA (even)
    GridReduce red_r;     // ||r||^2 per channel
    GridReduce red_b;     // ||b||^2 per channel (only if want_b)
    int want_b;
    int d_lo_zero;        // d.lo is all zero (FP32 data): its loads are skipped
};

// Staging layout of the refinement-residual kernel (dynamic shared memory,
// [slot][field][thread] for 128-thread CTAs: consecutive threads read
// consecutive 16-byte or 4-byte words, conflict-free). float4 fields per
// row: u.hi, u.lo, e, then d.hi, d.lo, y.hi, y.lo for RHS_SOURCE; word
// fields: the mask words of rows yb .. yb+RC, then per row the halo's mask
// word, u.hi, u.lo and e. The variants that read d only where a mask word
// says known (LOAD_D) are not staged: those loads depend on a word of the
// same chunk.
template <int RHS, int INIT, bool P32>
struct ResStage {
    static constexpr int RC = RES_CHUNK;
    static constexpr bool HAS_U = (INIT == INIT_KEEP || INIT == INIT_UPDATE);
    static constexpr bool HAS_E = (INIT == INIT_UPDATE || INIT == INIT_FROM32);
    static constexpr bool LOAD_D = (RHS == RHS_DATA) && (INIT != INIT_UPDATE);
    static constexpr bool STAGED = !LOAD_D;
    static constexpr int iUl = HAS_U ? 1 : 0;
    static constexpr int iE = iUl + ((HAS_U && !P32) ? 1 : 0);
    static constexpr int iD = iE + (HAS_E ? 1 : 0);
    static constexpr int NV = iD + (RHS == RHS_SOURCE ? 4 : 0);
    static constexpr int NSC = (RC + 1) + 4 * RC;
    // two chunks in flight ahead where 7 CTAs per SM still fit, else one
    static constexpr int NSLOT = (NV * RC <= 4) ? 3 : 2;
    static constexpr size_t bytes = STAGED ? (size_t)NSLOT * 128 * (NV * RC * 16 + NSC * 4) : 0;
};

// Quad strips like the FP32 kernels (lane = four columns, float4 loads of
// the hi and lo words). Known pixels take their Dirichlet value (d for
// RHS_DATA, 0 for RHS_SOURCE). With INIT_UPDATE the input iterate already
// holds it there (every refinement step writes it, and the V-cycle
// correction is zero on known pixels), so d is read only by the other INIT
// modes, once the row's mask word has arrived.
// Seven CTAs per SM (at most 72 registers). Launched with
// ResStage::bytes of dynamic shared memory, the loads of the next one or two
// chunks are in flight while a chunk is computed: each lane copies them
// (cp.async) into its own shared-memory slots and reads a chunk there once
// its copy group has landed -- the same addresses and the same arithmetic,
// so the results are bit-identical to the unstaged loop.
//
// P32 (plain FP32 form, RHS_DATA only): the iterate is a single FP32 word
// (the low words are neither read nor written), the update u + e and the
// stencil A u are plain FP32 operations. This is the per-image FP32 solver
// without iterative refinement that the mixed-precision path is compared
// against; its residual stalls near the FP32 rounding level.
template <int RHS, int INIT, bool P32>
__device__ __forceinline__ float2 residual_df_body(const ResArgs& a, int bx, int by, int ch) {
    static_assert(!P32 || RHS == RHS_DATA, "the plain FP32 form is an inpainting solve");
    constexpr int RC = RES_CHUNK;
    constexpr bool LOAD_D = (RHS == RHS_DATA) && (INIT != INIT_UPDATE);
    constexpr bool HAS_U = (INIT == INIT_KEEP || INIT == INIT_UPDATE);
    constexpr bool HAS_E = (INIT == INIT_UPDATE || INIT == INIT_FROM32);
    const MaskView m = a.m.ch(ch);
    const int H = a.F.H, W = a.F.W;
    const int y0 = (by * 4 + (threadIdx.x >> 5)) * a.rows;
    const int y1 = min(y0 + a.rows, H);
    pdl_trigger();
    const QuadLane q = quad_lane(bx * QS_COLS, a.F, m);
    const bool interior = bx > 0 && (bx + 1) * QS_COLS < W && y0 > 0 && y0 + a.rows + 1 <= H;
    pdl_wait();
    const int lane = q.lane;
    const long long co = ch * a.F.cs;
    float rr = 0.f, bb2 = 0.f;
    using SL = ResStage<RHS, INIT, P32>;
    constexpr int iUl = SL::iUl, iE = SL::iE, iD = SL::iD, NV = SL::NV, NSC = SL::NSC, NSLOT = SL::NSLOT;
    extern __shared__ float4 qs_dyn[];
    const bool staged = SL::STAGED && dyn_smem_bytes() >= SL::bytes;
    // slot sl, field f of this thread
    auto sv = [&](int sl, int f) { return qs_dyn + ((size_t)(sl * NV * RC + f) * 128 + threadIdx.x); };
    auto sw = [&](int sl, int f) {
        return reinterpret_cast<uint32_t*>(qs_dyn + (size_t)NSLOT * NV * RC * 128) +
               ((size_t)(sl * NSC + f) * 128 + threadIdx.x);
    };
    auto body = [&](auto in_tag) {
        constexpr bool IN = decltype(in_tag)::value;   // no border tests, no clamped rows
        const uint32_t* mrow = m.bits + q.mword;
        const uint32_t* hrow = m.bits + (q.hcol >> 5);
        const int hbit = q.hcol & 31;
        auto rowc = [&](int y) { return IN ? y : min(y, H - 1); };
        auto at = [&](int y, int col) { return co + (size_t)rowc(y) * a.F.pitch + col; };
        auto ld4 = [&](const float* p, size_t i) { return *reinterpret_cast<const float4*>(p + i); };
        // iterate value after the INIT transform, from the loaded sources
        auto value = [&](bool known, float uh, float ul, float e, float dh, float dl, float& h, float& l) {
            if (known) {
                if (RHS == RHS_DATA) {
                    if (INIT == INIT_UPDATE) { h = uh; l = ul; }
                    else { h = dh; l = dl; }
                } else {
                    h = 0.f; l = 0.f;
                }
            } else if (INIT == INIT_KEEP) {
                h = uh; l = ul;
            } else if (INIT == INIT_UPDATE) {
                if (P32) { h = uh + e; l = 0.f; }
                else df_add(uh, ul, e, 0.f, h, l);
            } else if (INIT == INIT_FROM32) {
                h = e; l = 0.f;
            } else {
                h = 0.f; l = 0.f;
            }
        };
        // the lane's four values of row y (all loads inside)
        auto row_value = [&](int y, float (&h)[4], float (&l)[4]) {
            const size_t i = at(y, q.cq);
            const uint32_t w = mrow[(size_t)rowc(y) * m.wpitch];
            float uh[4] = {0.f, 0.f, 0.f, 0.f}, ul[4] = {0.f, 0.f, 0.f, 0.f}, e[4] = {0.f, 0.f, 0.f, 0.f};
            float dh[4] = {0.f, 0.f, 0.f, 0.f}, dl[4] = {0.f, 0.f, 0.f, 0.f};
            if (HAS_U) {
                f4_to(ld4(a.uin.hi, i), uh);
                if (!P32) f4_to(ld4(a.uin.lo, i), ul);
            }
            if (HAS_E) f4_to(ld4(a.x32, i), e);
            if (LOAD_D) {
                f4_to(ld4(a.d.hi, i), dh);
                if (!a.d_lo_zero && !P32) f4_to(ld4(a.d.lo, i), dl);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) value((w >> (q.shift + j)) & 1u, uh[j], ul[j], e[j], dh[j], dl[j], h[j], l[j]);
        };
        float uph[4] = {0.f, 0.f, 0.f, 0.f}, upl[4] = {0.f, 0.f, 0.f, 0.f}, ch_[4], cl[4];
        row_value(y0, ch_, cl);
        if (IN || y0 > 0) row_value(y0 - 1, uph, upl);
        struct Chunk {
            float4 Uh[RC], Ul[RC], E[RC];          // rows yb+1 .. yb+RC
            float4 Dh[RC], Dl[RC], Yh[RC], Yl[RC];   // RHS_SOURCE: d and y of rows yb .. yb+RC-1
            float4 KDh[RC], KDl[RC];               // LOAD_D: data of rows yb+1 .. (known pixels)
            uint32_t Mw[RC + 1], Hm[RC];
            float HUh[RC], HUl[RC], HE[RC], HDh[RC], HDl[RC];   // halo column, rows yb ..
        };
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        auto load = [&](Chunk& c, int yb) {
#pragma unroll
            for (int k = 0; k <= RC; ++k) c.Mw[k] = mrow[(size_t)rowc(yb + k) * m.wpitch];
#pragma unroll
            for (int k = 0; k < RC; ++k) {
                const size_t id = at(yb + k + 1, q.cq), ih = at(yb + k, q.hcol), ic = at(yb + k, q.cq);
                c.Uh[k] = HAS_U ? ld4(a.uin.hi, id) : z4;
                c.Ul[k] = (HAS_U && !P32) ? ld4(a.uin.lo, id) : z4;
                c.E[k] = HAS_E ? ld4(a.x32, id) : z4;
                c.Hm[k] = q.hon ? hrow[(size_t)rowc(yb + k) * m.wpitch] : 0u;
                c.HUh[k] = (HAS_U && q.hon) ? a.uin.hi[ih] : 0.f;
                c.HUl[k] = (HAS_U && q.hon && !P32) ? a.uin.lo[ih] : 0.f;
                c.HE[k] = (HAS_E && q.hon) ? a.x32[ih] : 0.f;
                if (RHS == RHS_SOURCE) {
                    c.Dh[k] = ld4(a.d.hi, ic);
                    c.Dl[k] = a.d_lo_zero ? z4 : ld4(a.d.lo, ic);
                    c.Yh[k] = a.y.hi ? ld4(a.y.hi, ic) : z4;
                    c.Yl[k] = a.y.hi ? ld4(a.y.lo, ic) : z4;
                }
            }
            if (LOAD_D) {   // data only where the mask word says known
#pragma unroll
                for (int k = 0; k < RC; ++k) {
                    const uint32_t kb = (c.Mw[k + 1] >> q.shift) & 15u;
                    const size_t id = at(yb + k + 1, q.cq), ih = at(yb + k, q.hcol);
                    c.KDh[k] = kb ? ld4(a.d.hi, id) : z4;
                    c.KDl[k] = (kb && !a.d_lo_zero && !P32) ? ld4(a.d.lo, id) : z4;
                    const bool kh = q.hon && ((c.Hm[k] >> hbit) & 1u);
                    c.HDh[k] = kh ? a.d.hi[ih] : 0.f;
                    c.HDl[k] = (kh && !a.d_lo_zero && !P32) ? a.d.lo[ih] : 0.f;
                }
            }
        };
        // c: a Chunk in registers, or a StagedRows view of the staging slots
        auto compute = [&](const auto& c, int yb) {
#pragma unroll
            for (int k = 0; k < RC; ++k) {
                const int y = yb + k;
                if (!IN && y >= y1) break;
                float dnh[4] = {0.f, 0.f, 0.f, 0.f}, dnl[4] = {0.f, 0.f, 0.f, 0.f};
                if (IN || y + 1 < H) {
                    float uh[4], ul[4], e[4], dh[4], dl[4];
                    f4_to(c.Uh[k], uh);
                    f4_to(c.Ul[k], ul);
                    f4_to(c.E[k], e);
                    f4_to(LOAD_D ? c.KDh[k] : z4, dh);
                    f4_to(LOAD_D ? c.KDl[k] : z4, dl);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        value((c.Mw[k + 1] >> (q.shift + j)) & 1u, uh[j], ul[j], e[j], dh[j], dl[j], dnh[j], dnl[j]);
                }
                // horizontal neighbours outside the lane: shuffles, halo at the strip edges
                float lwh = __shfl_up_sync(HDI_FULL, ch_[3], 1), lwl = __shfl_up_sync(HDI_FULL, cl[3], 1);
                float rwh = __shfl_down_sync(HDI_FULL, ch_[0], 1), rwl = __shfl_down_sync(HDI_FULL, cl[0], 1);
                if (q.hon) {
                    float hh, hlo;
                    value((c.Hm[k] >> hbit) & 1u, c.HUh[k], c.HUl[k], c.HE[k], LOAD_D ? c.HDh[k] : 0.f,
                          LOAD_D ? c.HDl[k] : 0.f, hh, hlo);
                    if (lane == 0) { lwh = hh; lwl = hlo; }
                    else { rwh = hh; rwl = hlo; }
                }
                float sdh[4], sdl[4], syh[4], syl[4];
                if (RHS == RHS_SOURCE) {
                    f4_to(c.Dh[k], sdh);
                    f4_to(c.Dl[k], sdl);
                    f4_to(c.Yh[k], syh);
                    f4_to(c.Yl[k], syl);
                }
                float oh[4], ol[4], orr[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float cjh = ch_[j], cjl = cl[j];
                    oh[j] = cjh;
                    ol[j] = cjl;
                    const bool known = (c.Mw[k] >> (q.shift + j)) & 1u;
                    float r = 0.f;
                    if (known) {
                        if (RHS == RHS_DATA && (IN || q.act[j])) { const float bh = cjh + cjl; bb2 += bh * bh; }
                    } else {
                        // A u = 4 u_c - (sum of the 4 neighbours), an absent
                        // neighbour replaced by u_c (zero difference): the
                        // neighbour sum and the difference by TwoSum, the low
                        // parts added in FP32
                        const float lh = (j == 0) ? lwh : ch_[j - 1], ll = (j == 0) ? lwl : cl[j - 1];
                        const float rh = (j == 3) ? rwh : ch_[j + 1], rl = (j == 3) ? rwl : cl[j + 1];
                        const float n0h = (IN || q.lin[j]) ? lh : cjh, n0l = (IN || q.lin[j]) ? ll : cjl;
                        const float n1h = (IN || q.rin[j]) ? rh : cjh, n1l = (IN || q.rin[j]) ? rl : cjl;
                        const float n2h = (IN || y > 0) ? uph[j] : cjh, n2l = (IN || y > 0) ? upl[j] : cjl;
                        const float n3h = (IN || y + 1 < H) ? dnh[j] : cjh, n3l = (IN || y + 1 < H) ? dnl[j] : cjl;
                        if (P32) {   // plain FP32 stencil (b = 0 on unknown pixels)
                            r = -(4.f * cjh - ((n0h + n1h) + (n2h + n3h)));
                            orr[j] = r;
                            if (IN || q.act[j]) rr += r * r;
                            continue;
                        }
                        float sa, ea, sb, eb, sh, eh;
                        two_sum(n0h, n1h, sa, ea);
                        two_sum(n2h, n3h, sb, eb);
                        two_sum(sa, sb, sh, eh);
                        const float sl = ((n0l + n1l) + (n2l + n3l)) + ((ea + eb) + eh);
                        float ah, ae;
                        two_sum(4.f * cjh, -sh, ah, ae);
                        const float al = ae + (4.f * cjl - sl);   // A u = ah + al
                        if (RHS == RHS_SOURCE) {
                            float bh, bl;
                            df_add(sdh[j], sdl[j], -syh[j], -syl[j], bh, bl);
                            if (IN || q.act[j]) bb2 += bh * bh;
                            float rh2, rl2;
                            df_add(bh, bl, -ah, -al, rh2, rl2);
                            r = rh2 + rl2;
                        } else {
                            r = -(ah + al);   // b = 0 on unknown pixels
                        }
                    }
                    orr[j] = r;
                    if (IN || q.act[j]) rr += r * r;
                }
                const size_t idx = co + (size_t)y * a.F.pitch + q.c0;
                if (INIT == INIT_KEEP) {
                    // in place: only the known pixels change (to their
                    // Dirichlet value); readers take known pixels from d, so
                    // the order of these stores and their loads is immaterial
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if ((IN || q.act[j]) && ((c.Mw[k] >> (q.shift + j)) & 1u)) {
                            a.uout.hi[idx + j] = oh[j];
                            if (!P32) a.uout.lo[idx + j] = ol[j];
                        }
                    if (IN || q.act[3]) {
                        *reinterpret_cast<float4*>(a.r32 + idx) = make_float4(orr[0], orr[1], orr[2], orr[3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (q.act[j]) a.r32[idx + j] = orr[j];
                    }
                } else if (IN || q.act[3]) {
                    *reinterpret_cast<float4*>(a.uout.hi + idx) = make_float4(oh[0], oh[1], oh[2], oh[3]);
                    if (!P32) *reinterpret_cast<float4*>(a.uout.lo + idx) = make_float4(ol[0], ol[1], ol[2], ol[3]);
                    *reinterpret_cast<float4*>(a.r32 + idx) = make_float4(orr[0], orr[1], orr[2], orr[3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (q.act[j]) {
                            a.uout.hi[idx + j] = oh[j];
                            if (!P32) a.uout.lo[idx + j] = ol[j];
                            a.r32[idx + j] = orr[j];
                        }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    uph[j] = ch_[j]; upl[j] = cl[j];
                    ch_[j] = dnh[j]; cl[j] = dnl[j];
                }
            }
        };
        if (staged) {
            // copies of chunk yb into slot sl, from the addresses load() reads
            auto stage = [&](int sl, int yb) {
#pragma unroll
                for (int k = 0; k <= RC; ++k) cpa4(sw(sl, k), mrow + (size_t)rowc(yb + k) * m.wpitch);
#pragma unroll
                for (int k = 0; k < RC; ++k) {
                    const size_t id = at(yb + k + 1, q.cq), ih = at(yb + k, q.hcol), ic = at(yb + k, q.cq);
                    if (HAS_U) cpa16(sv(sl, k), a.uin.hi + id);
                    if (HAS_U && !P32) cpa16(sv(sl, iUl * RC + k), a.uin.lo + id);
                    if (HAS_E) cpa16(sv(sl, iE * RC + k), a.x32 + id);
                    if (RHS == RHS_SOURCE) {
                        cpa16(sv(sl, iD * RC + k), a.d.hi + ic);
                        if (!a.d_lo_zero) cpa16(sv(sl, (iD + 1) * RC + k), a.d.lo + ic);
                        if (a.y.hi) {
                            cpa16(sv(sl, (iD + 2) * RC + k), a.y.hi + ic);
                            cpa16(sv(sl, (iD + 3) * RC + k), a.y.lo + ic);
                        }
                    }
                    if (q.hon) {
                        cpa4(sw(sl, RC + 1 + k), hrow + (size_t)rowc(yb + k) * m.wpitch);
                        if (HAS_U) cpa4(sw(sl, RC + 1 + RC + k), a.uin.hi + ih);
                        if (HAS_U && !P32) cpa4(sw(sl, RC + 1 + 2 * RC + k), a.uin.lo + ih);
                        if (HAS_E) cpa4(sw(sl, RC + 1 + 3 * RC + k), a.x32 + ih);
                    }
                }
            };
            // the chunk as load() would have filled it, read where compute uses it
            auto view = [&](int sl) {
                StagedRows c;
                const float4* v = sv(sl, 0);
                const uint32_t* w = sw(sl, 0);
                c.Mw = {w, true};
                c.Uh = {v, HAS_U};
                c.Ul = {v + iUl * RC * 128, HAS_U && !P32};
                c.E = {v + iE * RC * 128, HAS_E};
                c.Dh = {v + iD * RC * 128, RHS == RHS_SOURCE};
                c.Dl = {v + (iD + 1) * RC * 128, RHS == RHS_SOURCE && !a.d_lo_zero};
                c.Yh = {v + (iD + 2) * RC * 128, RHS == RHS_SOURCE && a.y.hi != nullptr};
                c.Yl = {v + (iD + 3) * RC * 128, RHS == RHS_SOURCE && a.y.hi != nullptr};
                c.KDh = c.KDl = {v, false};
                c.Hm = {w + (RC + 1) * 128, q.hon};
                c.HUh = {w + (2 * RC + 1) * 128, HAS_U && q.hon};
                c.HUl = {w + (3 * RC + 1) * 128, HAS_U && q.hon && !P32};
                c.HE = {w + (4 * RC + 1) * 128, HAS_E && q.hon};
                c.HDh = c.HDl = {w, false};
                return c;
            };
            // slots in rotation; NSLOT - 1 chunks in flight ahead of the one computed
#pragma unroll
            for (int j = 0; j < NSLOT - 1; ++j) {
                if (y0 + j * RC < y1) stage(j, y0 + j * RC);
                cpa_commit();
            }
            int sl = 0;
            for (int yb = y0; yb < y1; yb += RC) {
                const int ya = yb + (NSLOT - 1) * RC;
                // slot of chunk ya: the one chunk yb - RC used (computed in the previous pass)
                if (ya < y1) stage(sl == 0 ? NSLOT - 1 : sl - 1, ya);
                cpa_commit();
                cpa_wait<NSLOT - 1>();   // chunk yb has landed
                compute(view(sl), yb);
                sl = (sl + 1 == NSLOT) ? 0 : sl + 1;
            }
        } else {
            for (int yb = y0; yb < y1; yb += RC) {
                Chunk A;
                load(A, yb);
                compute(A, yb);
            }
        }
    };
    if (interior) body(std::true_type{});
    else if (y0 < H) body(std::false_type{});
    return make_float2(rr, bb2);
}

template <int RHS, int INIT, bool P32 = false>
__global__ void __launch_bounds__(128, 7) k_residual_df(ResArgs a) {
    const float2 v = residual_df_body<RHS, INIT, P32>(a, blockIdx.x, blockIdx.y, blockIdx.z);
    const double tot = (double)block_sum_f(v.x);
    grid_reduce_commit(a.red_r, blockIdx.z, blockIdx.y * gridDim.x + blockIdx.x, tot);
    if (a.want_b) {
        const double totb = (double)block_sum_f(v.y);
        grid_reduce_commit(a.red_b, blockIdx.z, blockIdx.y * gridDim.x + blockIdx.x, totb);
    }
}

// One (image, channel) of a batched refinement-residual launch: ResArgs
// with the channel's planes (ch = 0) and its grid; the reductions of the
// ResArgs are unused (the batched launch commits to SegReduce).
struct ResTask {
    ResArgs a;
    int gx, gy;
};

// ||r||^2 of every task into red_r; with want_b also ||b||^2 into red_b (a
// second, same-shaped segmented reduction).
template <int RHS, int INIT, bool P32 = false>
__global__ void __launch_bounds__(128, 7) k_residual_df_b(const ResTask* __restrict__ tasks,
                                                       const int* __restrict__ cta0, int ntasks, SegReduce red_r,
                                                       SegReduce red_b, int want_b) {
    const int t = find_task(cta0, ntasks, blockIdx.x);
    const int local = blockIdx.x - cta0[t];
    const int gx = tasks[t].gx;
    const float2 v = residual_df_body<RHS, INIT, P32>(tasks[t].a, local % gx, local / gx, 0);
    const double tot = (double)block_sum_f(v.x);
    seg_reduce_commit(red_r, t, local, tot);
    if (want_b) {
        const double totb = (double)block_sum_f(v.y);
        seg_reduce_commit(red_b, t, local, totb);
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
                              T* __restrict__ dst, long long rs, long long cs, int c0) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int ch = blockIdx.z;
    if (x >= F.W) return;
    const size_t idx = ch * F.cs + (size_t)y * F.pitch + x;
    m = m.ch(c0 + ch);
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
    out[idx] = m.ch(ch).known(x, y) ? d.hi[idx] + d.lo[idx] : 0.f;
}

// ------------------------------------------------ batched FMG set-up ---

// One (image, channel) of the batched FMG data kernels: level geometry and
// mask plane, the channel's planes, and the task's blocks along x.
struct PixTask {
    LevelArr F, C;       // level (fine) and coarse level (data restriction)
    MaskView fm;         // mask plane of F
    DFc d;               // data on F (k_data_to_f32_b)
    const float* fb;     // FP32 data on F (k_restrict_data_b)
    float* out;          // output plane (on F for k_data_to_f32_b, on C for k_restrict_data_b)
    int gx;              // blocks along x
};

// Batched k_data_to_f32: 128 threads per block over 128 columns of one row.
__global__ void k_data_to_f32_b(const PixTask* __restrict__ tasks, const int* __restrict__ cta0, int ntasks) {
    const int t = find_task(cta0, ntasks, blockIdx.x);
    const int local = blockIdx.x - cta0[t];
    const PixTask& tk = tasks[t];
    const int x = (local % tk.gx) * blockDim.x + threadIdx.x;
    const int y = local / tk.gx;
    if (x >= tk.F.W || y >= tk.F.H) return;
    const size_t idx = (size_t)y * tk.F.pitch + x;
    tk.out[idx] = tk.fm.known(x, y) ? tk.d.hi[idx] + tk.d.lo[idx] : 0.f;
}

// Batched k_restrict_data: 32 x 8 threads per block over the coarse level.
__global__ void k_restrict_data_b(const PixTask* __restrict__ tasks, const int* __restrict__ cta0, int ntasks) {
    const int t = find_task(cta0, ntasks, blockIdx.x);
    const int local = blockIdx.x - cta0[t];
    const PixTask& tk = tasks[t];
    const int X = (local % tk.gx) * blockDim.x + threadIdx.x;
    const int Y = (local / tk.gx) * blockDim.y + threadIdx.y;
    if (X >= tk.C.W || Y >= tk.C.H) return;
    float s = 0.f;
    int n = 0;
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
            const int x = 2 * X + dx, y = 2 * Y + dy;
            if (x < tk.F.W && y < tk.F.H && tk.fm.known(x, y)) {
                s += tk.fb[(size_t)y * tk.F.pitch + x];
                ++n;
            }
        }
    tk.out[(size_t)Y * tk.C.pitch + X] = n ? s / (float)n : 0.f;
}

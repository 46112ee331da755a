// densify.cuh -- one Delaunay densification step (Sec. 4.1, Alg. 1) and the
// random-dithering initial mask (Sec. 4.2), on the GPU with exact integer
// geometry so that the new mask is reproducible bit for bit.
//
// Pipeline for a non-empty mask:
//   k_dens_error      e_p = sum_ch (u - f)^2 in FP64 (no contraction), and
//                     eq_p = rint(e_p * 2^20) for exact integer cell sums;
//   k_vor_columns     nearest known row above/below in each column (ties up);
//   k_vor_rows        exact Voronoi label: outward scan over columns with the
//                     per-column candidates, minimising (d^2, site index);
//   k_dens_quads      triangles of each 2x2 quad of labels (dual of the
//                     Voronoi diagram), collinear ones dropped, appended to a
//                     list with id 2*q + sub;
//   k_dens_raster     warp per triangle occurrence: every non-mask pixel
//                     centre inside the closed triangle takes atomicMin(id);
//                     duplicates of a triangle give the same pixels, so the
//                     owner ends up with the triangle's smallest id;
//   k_dens_cells      uncovered pixels join the hull cell of their label;
//                     E[cell] += eq (integer atomics: order-independent) and
//                     the largest e per cell (IEEE bits of e >= 0 are
//                     monotone as unsigned integers);
//   k_dens_argmax     lowest linear index among the pixels attaining it;
//   radix select      the k cells with the largest (E, -id) by 16-bit digit
//                     histograms; k_dens_commit sets their argmax pixels.
// An empty mask instead draws pixels with probability min(1, k w_i / sum w)
// from the Laplacian magnitude w (k_dens_lapw, k_dens_dither) and a
// counter-based SplitMix64 (Steele, Lea & Flood 2014).
#pragma once
#include "common.cuh"

// ------------------------------------------------------------ generator ---

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct DensImg {
    const double* f;   // [nch][H][W] FP64 copies of the caller data
    const double* u;
    int H, W, nch;
};

// w_i = sum_ch |(L f)_i|, neighbour differences added left, right, up, down;
// wq_i = rint(w_i * 2^24); sum of wq by integer atomics.
__global__ void k_dens_lapw(DensImg a, long long* __restrict__ wq, unsigned long long* total) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    long long q = 0;
    if (x < a.W) {
        double w = 0.0;
        const size_t n = (size_t)a.H * a.W;
        for (int ch = 0; ch < a.nch; ++ch) {
            const double* g = a.f + ch * n + (size_t)y * a.W;
            const double c = g[x];
            double acc = 0.0;
            if (x > 0) acc = __dadd_rn(acc, __dsub_rn(c, g[x - 1]));
            if (x + 1 < a.W) acc = __dadd_rn(acc, __dsub_rn(c, g[x + 1]));
            if (y > 0) acc = __dadd_rn(acc, __dsub_rn(c, g[x - a.W]));
            if (y + 1 < a.H) acc = __dadd_rn(acc, __dsub_rn(c, g[x + a.W]));
            w = __dadd_rn(w, fabs(acc));
        }
        q = __double2ll_rn(__dmul_rn(w, 16777216.0));
        wq[(size_t)y * a.W + x] = q;
    }
    unsigned long long s = (unsigned long long)q;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(HDI_FULL, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(total, s);
}

__global__ void k_dens_dither(const long long* __restrict__ wq, const unsigned long long* total, int H, int W,
                              long long k, uint64_t seed, uint8_t* __restrict__ mask, long long rs,
                              unsigned long long* added) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const size_t i = (size_t)y * W + x;
    const unsigned long long T = *total;
    double p;
    if (T > 0) p = fmin(1.0, __ddiv_rn(__dmul_rn((double)k, (double)wq[i]), __ull2double_rn(T)));
    else p = fmin(1.0, __ddiv_rn((double)k, (double)((long long)H * W)));
    const uint64_t h = splitmix64(seed, (uint64_t)i);
    if ((double)(h >> 11) < __dmul_rn(p, 9007199254740992.0)) {
        mask[(size_t)y * rs + x] = 1;
        atomicAdd(added, 1ull);
    }
}

// --------------------------------------------------------------- error ---

__global__ void k_dens_error(DensImg a, double* __restrict__ e, long long* __restrict__ eq) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.W) return;
    const size_t n = (size_t)a.H * a.W;
    const size_t i = (size_t)y * a.W + x;
    double s = 0.0;
    for (int ch = 0; ch < a.nch; ++ch) {
        const double d = __dsub_rn(a.u[ch * n + i], a.f[ch * n + i]);
        s = __dadd_rn(s, __dmul_rn(d, d));
    }
    e[i] = s;
    eq[i] = __double2ll_rn(__dmul_rn(s, 1048576.0));
}

// -------------------------------------------------------------- Voronoi ---

// Per column: the nearest known row to each row (ties to the upper row), or
// -1 if the column holds no known pixel. A block of 32 columns x 32 row
// segments: each thread scans its segment for its last and first known row,
// the segments' results meet in shared memory (the nearest known row above
// the segment is the last one of the nearest segment above that has one,
// likewise below), and each thread then walks its segment again to write
// the nearest row of every pixel. A warp reads one mask word per row and
// writes 32 consecutive columns.
constexpr int kVorSeg = 32;
__global__ void __launch_bounds__(32 * kVorSeg) k_vor_columns(MaskView m, int* __restrict__ ys) {
    __shared__ int lastk[kVorSeg][32], firstk[kVorSeg][32];
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int sg = threadIdx.y;
    const int len = (m.H + kVorSeg - 1) / kVorSeg;
    const int ya = min(sg * len, m.H), yb = min(ya + len, m.H);
    const bool col = x < m.W;
    int last = -1, first = -1;
    if (col)
        for (int y = ya; y < yb; ++y)
            if (m.known(x, y)) {
                if (first < 0) first = y;
                last = y;
            }
    lastk[sg][threadIdx.x] = last;
    firstk[sg][threadIdx.x] = first;
    __syncthreads();
    if (!col) return;
    int up = -1;   // nearest known row above the segment
    for (int t = sg - 1; t >= 0 && up < 0; --t) up = lastk[t][threadIdx.x];
    int next = -1;   // nearest known row below the segment
    for (int t = sg + 1; t < kVorSeg && next < 0; ++t) next = firstk[t][threadIdx.x];
    // downward: nearest known row at or above y
    for (int y = ya; y < yb; ++y) {
        if (m.known(x, y)) up = y;
        ys[(size_t)y * m.W + x] = up;
    }
    // upward: combine with the nearest known row at or below y
    for (int y = yb - 1; y >= ya; --y) {
        if (m.known(x, y)) next = y;
        const size_t i = (size_t)y * m.W + x;
        const int u = ys[i];
        int best;
        if (u < 0) best = next;
        else if (next < 0) best = u;
        else best = (y - u <= next - y) ? u : next;
        ys[i] = best;
    }
}

// The launch shape k_vor_columns is written for (32 columns x kVorSeg row
// segments per block); every caller goes through this.
inline void launch_vor_columns(const MaskView& m, int* ys, cudaStream_t s) {
    k_vor_columns<<<(m.W + 31) / 32, dim3(32, kVorSeg), 0, s>>>(m, ys);
}

// Exact label: minimise (d^2, linear index of the site) over all columns,
// scanning outward from x until dx^2 exceeds the best d^2.
__global__ void k_vor_rows(const int* __restrict__ ys, int H, int W, int* __restrict__ V) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const int* row = ys + (size_t)y * W;
    long long bd = LLONG_MAX;
    long long bs = LLONG_MAX;
    for (int dx = 0; dx < W; ++dx) {
        const long long dx2 = (long long)dx * dx;
        if (dx2 > bd) break;
        for (int side = 0; side < (dx ? 2 : 1); ++side) {
            const int xx = side ? x + dx : x - dx;
            if (xx < 0 || xx >= W) continue;
            const int yy = row[xx];
            if (yy < 0) continue;
            const long long d2 = dx2 + (long long)(y - yy) * (y - yy);
            const long long s = (long long)yy * W + xx;
            if (d2 < bd || (d2 == bd && s < bs)) { bd = d2; bs = s; }
        }
    }
    V[(size_t)y * W + x] = (int)bs;
}

// Jump flooding (Rong and Tan 2006), the paper's approximate Voronoi diagram
// (Sec. 4.2): seeds label themselves; each pass with step k gives every pixel
// the site of least (d^2, linear index) among its own label and those of the
// 8 pixels at offsets (+-k or 0, +-k or 0) in the previous pass.
__global__ void k_jfa_init(MaskView m, int* __restrict__ lab) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= m.W) return;
    const size_t p = (size_t)y * m.W + x;
    lab[p] = m.known(x, y) ? (int)p : -1;
}

__global__ void k_jfa_pass(const int* __restrict__ in, int* __restrict__ out, int H, int W, int k) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    long long bd = LLONG_MAX;
    int bs = -1;
    for (int dy = -k; dy <= k; dy += k) {
        const int ny = y + dy;
        if (ny < 0 || ny >= H) continue;
        for (int dx = -k; dx <= k; dx += k) {
            const int nx = x + dx;
            if (nx < 0 || nx >= W) continue;
            const int s = in[(size_t)ny * W + nx];
            if (s < 0) continue;
            const int sy = s / W, sx = s - sy * W;
            const long long d2 = (long long)(x - sx) * (x - sx) + (long long)(y - sy) * (y - sy);
            if (d2 < bd || (d2 == bd && s < bs)) { bd = d2; bs = s; }
        }
    }
    out[(size_t)y * W + x] = bs;
}

// Largest squared pixel-to-site distance of a label map (the bound that lets
// the next, denser mask start jump flooding with a smaller step); all ones if
// a pixel has no label.
__global__ void k_label_maxd2(const int* __restrict__ V, int H, int W, unsigned long long* maxd2) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    unsigned long long d2 = 0;
    if (x < W) {
        const int s = V[(size_t)y * W + x];
        if (s < 0) {
            d2 = ~0ull;   // unlabelled pixel
        } else {
            const int sy = s / W, sx = s - sy * W;
            d2 = (unsigned long long)((long long)(x - sx) * (x - sx) + (long long)(y - sy) * (y - sy));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(HDI_FULL, d2, o);
        d2 = v > d2 ? v : d2;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(maxd2, d2);
}

// ------------------------------------------------------------ triangles ---

struct Tri {
    int v[3];
    int id;
};

__device__ __forceinline__ long long orient2(long long ax, long long ay, long long bx, long long by, long long cx,
                                             long long cy) {
    return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
}

// Appends of one warp's triangles (0, 1 or 2 per thread) with one atomic
// per warp: the list order is immaterial (ownership takes the minimum id).
__device__ __forceinline__ void push_tris(const Tri (&t)[2], int n, Tri* list, unsigned* count, unsigned cap) {
    const int lane = threadIdx.x & 31;
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(HDI_FULL, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(HDI_FULL, incl, 31);
    unsigned base = 0;
    if (lane == 31 && total) base = atomicAdd(count, (unsigned)total);
    base = __shfl_sync(HDI_FULL, base, 31);
    const unsigned slot = base + (unsigned)(incl - n);
    for (int k = 0; k < n; ++k)
        if (slot + k < cap) list[slot + k] = t[k];
}

__device__ __forceinline__ void add_tri(Tri (&t)[2], int& n, int a, int b, int c, int id, int W) {
    if (orient2(a % W, a / W, b % W, b / W, c % W, c / W) == 0) return;   // collinear: dropped
    t[n].v[0] = a;
    t[n].v[1] = b;
    t[n].v[2] = c;
    t[n].id = id;
    ++n;
}

__global__ void k_dens_quads(const int* __restrict__ V, int H, int W, Tri* __restrict__ list, unsigned* count,
                             unsigned cap) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    Tri t[2];
    int n = 0;
    if (x < W - 1 && y < H - 1) {
        const int a = V[(size_t)y * W + x];          // TL
        const int b = V[(size_t)y * W + x + 1];      // TR
        const int c = V[(size_t)(y + 1) * W + x + 1];// BR
        const int d = V[(size_t)(y + 1) * W + x];    // BL
        const int q = y * (W - 1) + x;
        const bool ab = a == b, ac = a == c, ad = a == d, bc = b == c, bd = b == d, cd = c == d;
        const int pairs = ab + ac + ad + bc + bd + cd;
        if (pairs == 0) {   // four distinct sites in cyclic order a, b, c, d
            add_tri(t, n, a, b, c, 2 * q, W);
            add_tri(t, n, a, c, d, 2 * q + 1, W);
        } else if (pairs == 1) {   // exactly three distinct sites
            int s1, s2;
            if (ab) { s1 = c; s2 = d; }
            else if (ac) { s1 = b; s2 = d; }
            else if (ad) { s1 = b; s2 = c; }
            else if (bc) { s1 = b; s2 = d; }
            else if (bd) { s1 = b; s2 = c; }
            else { s1 = b; s2 = c; }   // cd
            add_tri(t, n, a, s1, s2, 2 * q, W);
        }
    }
    push_tris(t, n, list, count, cap);
}

// Warp per triangle occurrence: closed-triangle containment by integer
// orientation tests; atomicMin of the id on non-mask pixels.
__global__ void k_dens_raster(const Tri* __restrict__ list, const unsigned* count, MaskView m,
                              int* __restrict__ owner) {
    const unsigned t = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= *count) return;
    const Tri tr = list[t];
    const int W = m.W;
    long long ax = tr.v[0] % W, ay = tr.v[0] / W;
    long long bx = tr.v[1] % W, by = tr.v[1] / W;
    long long cx = tr.v[2] % W, cy = tr.v[2] / W;
    if (orient2(ax, ay, bx, by, cx, cy) < 0) {
        long long tx = bx, ty = by;
        bx = cx; by = cy; cx = tx; cy = ty;
    }
    const long long x0 = min(ax, min(bx, cx)), x1 = max(ax, max(bx, cx));
    const long long y0 = min(ay, min(by, cy)), y1 = max(ay, max(by, cy));
    const long long bw = x1 - x0 + 1;
    const long long n = bw * (y1 - y0 + 1);
    for (long long i = lane; i < n; i += 32) {
        const long long px = x0 + i % bw, py = y0 + i / bw;
        if (orient2(ax, ay, bx, by, px, py) >= 0 && orient2(bx, by, cx, cy, px, py) >= 0 &&
            orient2(cx, cy, ax, ay, px, py) >= 0) {
            if (!m.known((int)px, (int)py)) atomicMin(owner + py * W + px, tr.id);
        }
    }
}

constexpr int kNoOwner = 0x7F7F7F7F;   // memset(0x7F) sentinel, above every cell id

// Hull cells, cell sums and the per-cell maximum of e.
__global__ void k_dens_cells(MaskView m, const int* __restrict__ V, int* __restrict__ owner,
                             const long long* __restrict__ eq, const double* __restrict__ e,
                             unsigned long long* __restrict__ E, unsigned long long* __restrict__ emax,
                             int hull_base) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= m.W) return;
    const size_t i = (size_t)y * m.W + x;
    if (m.known(x, y)) {
        owner[i] = -1;
        return;
    }
    int o = owner[i];
    if (o == kNoOwner) {
        o = hull_base + V[i];
        owner[i] = o;
    }
    if (eq[i]) atomicAdd(E + o, (unsigned long long)eq[i]);
    atomicMax(emax + o, (unsigned long long)__double_as_longlong(e[i]));
}

__global__ void k_dens_argmax(MaskView m, const int* __restrict__ owner, const double* __restrict__ e,
                              const unsigned long long* __restrict__ emax, int* __restrict__ arg) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= m.W) return;
    const size_t i = (size_t)y * m.W + x;
    const int o = owner[i];
    if (o < 0) return;
    if ((unsigned long long)__double_as_longlong(e[i]) == emax[o]) atomicMin(arg + o, (int)i);
}

// ------------------------------------------------------------ selection ---

// Candidate list: cells with E > 0.
// Candidate list (cells with E > 0) in any order (the selection depends on
// the keys only), and the largest E (emax), which gives the selection its
// highest nonzero digit. A block of 256 threads scans 2048 cells (eight per
// thread, coalesced): one atomic per block for its slots, and the maximum
// only when the block's exceeds the value already stored.
constexpr int kCandPer = 8;
__global__ void __launch_bounds__(256) k_dens_candidates(const unsigned long long* __restrict__ E, int ncell,
                                                         int* __restrict__ cand, unsigned* ncand,
                                                         unsigned long long* emax) {
    __shared__ unsigned wsum[8];
    __shared__ unsigned long long wmax[8];
    __shared__ unsigned base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long b0 = (long long)blockIdx.x * (256 * kCandPer);
    unsigned long long e[kCandPer];
    unsigned n = 0;
    unsigned long long m = 0;
#pragma unroll
    for (int k = 0; k < kCandPer; ++k) {
        const long long i = b0 + k * 256 + threadIdx.x;
        e[k] = (i < ncell) ? E[i] : 0ull;
        n += e[k] != 0;
        m = e[k] > m ? e[k] : m;
    }
    // exclusive prefix of n over the block: warp scan, then the warp totals
    unsigned incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(HDI_FULL, incl, o);
        if (lane >= o) incl += v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(HDI_FULL, m, o);
        m = v > m ? v : m;
    }
    if (lane == 31) wsum[wid] = incl;
    if (lane == 0) wmax[wid] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned tot = 0;
        unsigned long long bm = 0;
        for (int w = 0; w < 8; ++w) {
            const unsigned t = wsum[w];
            wsum[w] = tot;
            tot += t;
            bm = wmax[w] > bm ? wmax[w] : bm;
        }
        base = tot ? atomicAdd(ncand, tot) : 0u;
        if (bm > *(volatile unsigned long long*)emax) atomicMax(emax, bm);
    }
    __syncthreads();
    unsigned slot = base + wsum[wid] + incl - n;
#pragma unroll
    for (int k = 0; k < kCandPer; ++k)
        if (e[k]) cand[slot++] = (int)(b0 + k * 256 + threadIdx.x);
}

// Histogram of one 16-bit digit of the key among candidates whose higher
// digits equal `prefix`. Key = E (mode 0) or the cell id among E == tieE
// (mode 1). Lanes of a warp with the same bin add once (the keys of a
// selection concentrate in few bins).
__global__ void k_dens_hist(const int* __restrict__ cand, const unsigned* ncand,
                            const unsigned long long* __restrict__ E, int mode, unsigned long long tieE,
                            int shift, unsigned long long prefix, unsigned* __restrict__ hist) {
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned bin = 0xFFFFFFFFu;   // no contribution
    if (i < *ncand) {
        const int c = cand[i];
        unsigned long long key = 0;
        bool ok = true;
        if (mode == 0) key = E[c];
        else {
            ok = E[c] == tieE;
            key = (unsigned long long)c;
        }
        const unsigned long long hi = (shift + 16 >= 64) ? 0ull : (key >> (shift + 16));
        if (ok && hi == prefix) bin = (unsigned)((key >> shift) & 0xFFFFull);
    }
    const unsigned same = __match_any_sync(HDI_FULL, bin);
    const int lane = threadIdx.x & 31;
    if (bin != 0xFFFFFFFFu && lane == __ffs(same) - 1) atomicAdd(hist + bin, (unsigned)__popc(same));
}

// Select cells with E > T, or E == T and id <= Tid; set their argmax pixel.
__global__ void k_dens_commit(const int* __restrict__ cand, const unsigned* ncand,
                              const unsigned long long* __restrict__ E, unsigned long long T, long long Tid,
                              const int* __restrict__ arg, int W, uint8_t* __restrict__ mask, long long rs,
                              unsigned long long* added) {
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    bool sel = false;
    if (i < *ncand) {
        const int c = cand[i];
        const unsigned long long ec = E[c];
        if (ec > T || (ec == T && (long long)c <= Tid)) {
            const int p = arg[c];
            mask[(size_t)(p / W) * rs + p % W] = 1;
            sel = true;
        }
    }
    const unsigned ball = __ballot_sync(HDI_FULL, sel);
    if ((threadIdx.x & 31) == 0 && ball) atomicAdd(added, (unsigned long long)__popc(ball));
}

// Plain FP64 copy of a caller image (any strides) into [nch][H][W].
template <typename T>
__global__ void k_dens_load(const T* __restrict__ src, long long rs, long long cs, int H, int W,
                            double* __restrict__ dst) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int ch = blockIdx.z;
    if (x >= W) return;
    dst[(size_t)ch * H * W + (size_t)y * W + x] = (double)src[ch * cs + (size_t)y * rs + x];
}

// ------------------------------------------------------- host-side loop ---

// Copies a caller image (device or host) into a plain FP64 [nch][H][W] array.
int Ctx::dens_load(const hdi_image* im, double* dst, void* hstage) {
    const void* src = im->data;
    long long rs = im->row_stride, cs = im->channel_stride;
    const size_t es = im->dtype == HDI_F64 ? 8 : 4;
    if (im->location == HDI_HOST) {
        for (int c = 0; c < nch; ++c) {
            cudaError_t e = cudaMemcpy2DAsync((char*)hstage + (size_t)c * H * W * es, W * es,
                                              (const char*)src + (size_t)c * cs * es, rs * es, W * es, H,
                                              cudaMemcpyHostToDevice, stream);
            if (e != cudaSuccess) return cuda_check(e, "host-to-device copy");
        }
        src = hstage;
        rs = W;
        cs = (long long)H * W;
    }
    dim3 grd((W + 127) / 128, H, nch);
    if (im->dtype == HDI_F64) k_dens_load<double><<<grd, 128, 0, stream>>>((const double*)src, rs, cs, H, W, dst);
    else k_dens_load<float><<<grd, 128, 0, stream>>>((const float*)src, rs, cs, H, W, dst);
    ++launches;
    return HDI_OK;
}

int Ctx::densify(const hdi_image* f, hdi_mask* mask, const hdi_image* u, int64_t k, uint64_t seed, int64_t* added) {
    int rc;
    if ((rc = cuda_check(cudaSetDevice(device), "cudaSetDevice"))) return rc;
    if (!added) return fail(HDI_ERR_INVALID_ARG, "added: null");
    *added = 0;
    if ((rc = check_image(f, "f", -1, 0, 0))) return rc;
    if (k < 0) return fail(HDI_ERR_INVALID_ARG, "k must be >= 0");
    if (u && (rc = check_image(u, "u", f->height, f->width, f->channels))) return rc;
    if ((rc = setup(f->height, f->width, f->channels))) return rc;
    long long ones = 0;
    if ((rc = load_mask(mask, &ones))) return rc;
    uint8_t* mptr = mask->data;
    long long mrs = mask->row_stride;
    if (mask->location == HDI_HOST) {
        mptr = (uint8_t*)stage.base + (size_t)nch * H * W * 8;   // staged by load_mask
        mrs = W;
    }
    if (ones > 0 && !u) return fail(HDI_ERR_INVALID_ARG, "u: required when the mask is not empty");
    const size_t N = (size_t)H * W;
    const int hull_base = 2 * (W - 1) * (H - 1);
    const size_t ncell = (size_t)hull_base + N + 1;
    const size_t tcap = (size_t)2 * (W > 1 ? W - 1 : 1) * (H > 1 ? H - 1 : 1) + 16;
    // layout
    size_t bytes = 0;
    auto acc = [&](size_t b) { bytes += (b + 255) & ~(size_t)255; };
    const size_t sizes[] = {(size_t)nch * N * 8, (size_t)nch * N * 8, (size_t)nch * N * 8, N * 8, N * 8, N * 4, N * 4,
                            N * 4, tcap * sizeof(Tri), ncell * 8, ncell * 8, ncell * 4, ncell * 4, 65536 * 4, 256};
    for (size_t s : sizes) acc(s);
    if ((rc = dws.reserve(*this, std::max(dws.cap, bytes), "densification workspace"))) return rc;
    double* F = (double*)dws.take(sizes[0]);
    double* Uu = (double*)dws.take(sizes[1]);
    void* hst = dws.take(sizes[2]);
    double* e = (double*)dws.take(sizes[3]);
    long long* eq = (long long*)dws.take(sizes[4]);
    int* ys = (int*)dws.take(sizes[5]);
    int* V = (int*)dws.take(sizes[6]);
    int* owner = (int*)dws.take(sizes[7]);
    Tri* tris = (Tri*)dws.take(sizes[8]);
    unsigned long long* E = (unsigned long long*)dws.take(sizes[9]);
    unsigned long long* emax = (unsigned long long*)dws.take(sizes[10]);
    int* arg = (int*)dws.take(sizes[11]);
    int* cand = (int*)dws.take(sizes[12]);
    unsigned* hist = (unsigned*)dws.take(sizes[13]);
    unsigned long long* cnt = (unsigned long long*)dws.take(sizes[14]);   // [0] added, [1] total, [2..] counts
    if (dws.used > dws.cap) return fail(HDI_ERR_CUDA, "internal: densification workspace carving exceeds its reservation");
    cudaMemsetAsync(cnt, 0, 256, stream);
    if ((rc = dens_load(f, F, hst))) return rc;
    DensImg img;
    img.f = F;
    img.u = Uu;
    img.H = H;
    img.W = W;
    img.nch = nch;
    dim3 grow((W + 127) / 128, H);
    unsigned long long hcnt[6] = {0, 0, 0, 0, 0, 0};
    if (ones == 0) {
        long long* wq = eq;   // reuse
        k_dens_lapw<<<grow, 128, 0, stream>>>(img, wq, cnt + 1);
        k_dens_dither<<<grow, 128, 0, stream>>>(wq, cnt + 1, H, W, (long long)k, seed, mptr, mrs, cnt);
        launches += 2;
    } else {
        if ((rc = dens_load(u, Uu, hst))) return rc;
        const MaskView mv = mview(0);
        k_dens_error<<<grow, 128, 0, stream>>>(img, e, eq);
        if (p.densify_voronoi >= 0.5) {
            // jump flooding from the first step, ping-pong between ys and V so
            // that the last pass lands in V
            int full = 1;
            while (full < std::max(H, W)) full *= 2;
            full = std::max(full / 2, 1);
            int first = (int)p.jfa_first_step;
            if (first < 1 || first > full) first = full;
            for (;;) {
                int passes = 0;
                for (int k2 = first; k2 >= 1; k2 /= 2) ++passes;
                int* a0 = (passes & 1) ? ys : V;
                int* a1 = (passes & 1) ? V : ys;
                k_jfa_init<<<grow, 128, 0, stream>>>(mv, a0);
                ++launches;
                for (int k2 = first; k2 >= 1; k2 /= 2) {
                    k_jfa_pass<<<grow, 128, 0, stream>>>(a0, a1, H, W, k2);
                    ++launches;
                    std::swap(a0, a1);
                }
                if (first == full) break;
                // a shortened schedule must still reach every pixel; if it
                // did not, run the full one
                cudaMemsetAsync(cnt + 4, 0, 8, stream);
                k_label_maxd2<<<grow, 128, 0, stream>>>(V, H, W, cnt + 4);
                ++launches;
                unsigned long long md = 0;
                cudaMemcpyAsync(&md, cnt + 4, 8, cudaMemcpyDeviceToHost, stream);
                if ((rc = sync("jump flooding"))) return rc;
                if (md != ~0ull) break;
                first = full;
            }
        } else {
            launch_vor_columns(mv, ys, stream);
            k_vor_rows<<<grow, 128, 0, stream>>>(ys, H, W, V);
            launches += 2;
        }
        // the labels' largest distance bounds the next jump-flooding schedule
        // (hdi_densify with densify_voronoi = 1); exact labels need none
        cudaMemsetAsync(cnt + 4, 0, 8, stream);
        if (p.densify_voronoi >= 0.5) {
            k_label_maxd2<<<grow, 128, 0, stream>>>(V, H, W, cnt + 4);
            ++launches;
        }
        unsigned* tcount = (unsigned*)(cnt + 2);
        unsigned* ncand = (unsigned*)(cnt + 3);
        // Voronoi-cell partition (densify_partition = 1): no triangles; every
        // non-mask pixel falls to the "hull" cell of its label below, whose
        // id hull_base + V(p) ranks like the site index V(p)
        const bool vcells = p.densify_partition >= 0.5;
        if (!vcells) {
            k_dens_quads<<<dim3((W + 127) / 128, H), 128, 0, stream>>>(V, H, W, tris, tcount, (unsigned)tcap);
            ++launches;
        }
        cudaMemsetAsync(owner, 0x7F, N * 4, stream);
        ++launches;   // k_dens_error
        cudaMemcpyAsync(hcnt, cnt, 40, cudaMemcpyDeviceToHost, stream);
        if ((rc = sync("densification triangles"))) return rc;
        last_label_maxd2 = (long long)hcnt[4];
        const unsigned ntri = vcells ? 0u : (unsigned)(hcnt[2] & 0xffffffffull);
        if (ntri > tcap) return fail(HDI_ERR_CUDA, "internal: triangle list overflow");
        if (ntri) {
            k_dens_raster<<<(ntri + 3) / 4, 128, 0, stream>>>(tris, tcount, mv, owner);
            ++launches;
        }
        cudaMemsetAsync(E, 0, ncell * 8, stream);
        cudaMemsetAsync(emax, 0, ncell * 8, stream);
        cudaMemsetAsync(arg, 0x7F, ncell * 4, stream);
        k_dens_cells<<<grow, 128, 0, stream>>>(mv, V, owner, eq, e, E, emax, hull_base);
        k_dens_argmax<<<grow, 128, 0, stream>>>(mv, owner, e, emax, arg);
        k_dens_candidates<<<(unsigned)((ncell + 256 * kCandPer - 1) / (256 * kCandPer)), 256, 0, stream>>>(
            E, (int)ncell, cand, ncand, cnt + 5);
        launches += 3;
        cudaMemcpyAsync(hcnt, cnt, 48, cudaMemcpyDeviceToHost, stream);
        if ((rc = sync("densification cells"))) return rc;
        const unsigned nc = (unsigned)(hcnt[3] & 0xffffffffull);
        unsigned long long T = 0;
        long long Tid = -1;
        if (nc > (unsigned long long)k) {
            // radix select of the k-th largest E (16-bit digits, most significant first)
            std::vector<unsigned> h(65536);
            unsigned long long need = (unsigned long long)k, prefix = 0;
            const unsigned blocks = (nc + 255) / 256;
            // digits above the largest E are 0 for every key: start below them
            const unsigned long long emax_h = hcnt[5];
            int top = 0;
            while (top < 48 && (emax_h >> (top + 16)) != 0) top += 16;
            for (int shift = top; shift >= 0 && need > 0; shift -= 16) {
                cudaMemsetAsync(hist, 0, 65536 * 4, stream);
                k_dens_hist<<<blocks, 256, 0, stream>>>(cand, ncand, E, 0, 0, shift, prefix, hist);
                ++launches;
                cudaMemcpyAsync(h.data(), hist, 65536 * 4, cudaMemcpyDeviceToHost, stream);
                if ((rc = sync("densification selection"))) return rc;
                unsigned long long cum = 0;
                int dsel = 0;
                for (int dgt = 65535; dgt >= 0; --dgt) {
                    if (cum + h[dgt] >= need) { dsel = dgt; break; }
                    cum += h[dgt];
                }
                need -= cum;
                prefix = (prefix << 16) | (unsigned long long)dsel;
            }
            T = prefix;
            // among E == T keep the `need` smallest ids
            unsigned long long pid = 0;
            for (int shift = 16; shift >= 0; shift -= 16) {
                cudaMemsetAsync(hist, 0, 65536 * 4, stream);
                k_dens_hist<<<blocks, 256, 0, stream>>>(cand, ncand, E, 1, T, shift, pid, hist);
                ++launches;
                cudaMemcpyAsync(h.data(), hist, 65536 * 4, cudaMemcpyDeviceToHost, stream);
                if ((rc = sync("densification tie break"))) return rc;
                unsigned long long cum = 0;
                int dsel = 0;
                for (int dgt = 0; dgt < 65536; ++dgt) {
                    if (cum + h[dgt] >= need) { dsel = dgt; break; }
                    cum += h[dgt];
                }
                need -= cum;
                pid = (pid << 16) | (unsigned long long)dsel;
            }
            Tid = (long long)pid;
        }
        if (nc && k > 0) {
            k_dens_commit<<<(nc + 255) / 256, 256, 0, stream>>>(cand, ncand, E, T, Tid, arg, W, mptr, mrs, cnt);
            ++launches;
        }
    }
    cudaMemcpyAsync(hcnt, cnt, 32, cudaMemcpyDeviceToHost, stream);
    if ((rc = sync("densification"))) return rc;
    *added = (int64_t)hcnt[0];
    if (mask->location == HDI_HOST) {
        cudaError_t ce = cudaMemcpy2DAsync(mask->data, mask->row_stride, mptr, W, W, H, cudaMemcpyDeviceToHost, stream);
        if (ce != cudaSuccess) return cuda_check(ce, "mask download");
        if ((rc = sync("mask download"))) return rc;
    }
    return HDI_OK;
}

// common.cuh -- shared device helpers of libhdi (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define HDI_FULL 0xffffffffu

// Bit-packed mask: one uint32 word per 32 pixels along x, `wpitch` words per
// row (ceil(W/32) + 1; the extra zero word lets a 32-wide window starting at
// any x read two words without a bounds check). Bit set = known pixel (c = 1).
struct MaskView {
    const uint32_t* bits;
    int H, W, wpitch;
    // Batched solves give every channel its own mask plane: channel c uses
    // plane chmask[c], `cstride` words apart. chmask == nullptr: one mask
    // shared by all channels (Sec. 2.1).
    const int* chmask;
    long long cstride;
    __device__ __forceinline__ MaskView ch(int c) const {
        MaskView r = *this;
        if (chmask) r.bits += (size_t)chmask[c] * cstride;
        return r;
    }
    __device__ __forceinline__ bool known(int x, int y) const {
        return (bits[(size_t)y * wpitch + (x >> 5)] >> (x & 31)) & 1u;
    }
    // 32 mask bits for columns x0 .. x0+31 of row y (bit i = column x0+i).
    __device__ __forceinline__ uint32_t window(int x0, int y) const {
        const uint32_t* row = bits + (size_t)y * wpitch + (x0 >> 5);
        return __funnelshift_r(row[0], row[1], x0 & 31);
    }
};

// Programmatic dependent launch (sm_90 and later). The multigrid kernels are
// launched with programmatic stream serialisation: a kernel's CTAs may be
// scheduled while its predecessor in the stream is still finishing, run the
// part that reads only launch arguments and the mask (unchanged during a
// solve), and then wait in pdl_wait() until the predecessor grid has
// completed and its writes are visible. pdl_trigger() at a kernel's start
// lets its own successor be scheduled early. Launched without the attribute,
// both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Lane-private asynchronous staging (cp.async): a thread copies global words
// into shared-memory slots that only it reads, then waits for its own copy
// groups. No other thread touches the slots, so no barrier is needed, and
// the wait is the hardware's group wait (no polling loop). The streaming
// stencil kernels use it to keep the next rows' loads in flight while they
// compute the current ones, without a second register buffer. 16-byte copies
// need 16-byte aligned source and destination.
__device__ __forceinline__ void cpa16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cpa4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
// Dynamic shared memory given to this launch, in bytes: a kernel stages its
// loads only when the launch provided the slots its layout needs.
__device__ __forceinline__ unsigned dyn_smem_bytes() {
    unsigned r;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's copy groups are still in flight
template <int N>
__device__ __forceinline__ void cpa_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(HDI_FULL, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(HDI_FULL, v, o);
    return v;
}

__device__ __forceinline__ int linear_tid() {
    return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
}

// Block-wide FP64 sum in a fixed tree order; result valid in thread 0.
// All threads of the block must call it.
__device__ __forceinline__ double block_sum_d(double v) {
    __shared__ double sh[32];
    const int tid = linear_tid();
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    v = warp_sum_d(v);
    __syncthreads();
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    const int nw = (nt + 31) >> 5;
    v = (tid < nw) ? sh[tid] : 0.0;
    if (tid < 32) v = warp_sum_d(v);
    return v;
}

// Block-wide FP32 sum in a fixed tree order; result valid in thread 0.
// (Per-pixel reductions run in FP32: the FP64 pipe of the target is a small
// fraction of its FP32 pipe. Only one FP64 value per CTA reaches the grid
// reduction.)
__device__ __forceinline__ float block_sum_f(float v) {
    __shared__ float shf[32];
    const int tid = linear_tid();
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    v = warp_sum_f(v);
    __syncthreads();
    if ((tid & 31) == 0) shf[tid >> 5] = v;
    __syncthreads();
    const int nw = (nt + 31) >> 5;
    v = (tid < nw) ? shf[tid] : 0.f;
    if (tid < 32) v = warp_sum_f(v);
    return v;
}

// Deterministic grid reduction: every CTA deposits one FP64 partial per
// (channel, part); the last CTA to arrive sums each channel's partials in a
// fixed order and writes out[ch]. `nparts` CTAs per channel, `nch` channels;
// all nparts*nch CTAs of the launch call grid_reduce_commit exactly once.
struct GridReduce {
    double* partials;   // [nch * nparts]
    double* out;        // [nch]
    unsigned* ticket;   // zero before the launch; reset to zero by the last CTA
    int nparts;
    int nch;
};

__device__ __forceinline__ void grid_reduce_commit(const GridReduce& R, int ch, int part, double block_total) {
    __shared__ bool last_cta;
    const int tid = linear_tid();
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    if (tid == 0) {
        R.partials[(size_t)ch * R.nparts + part] = block_total;
        __threadfence();
        unsigned t = atomicAdd(R.ticket, 1u);
        last_cta = (t == (unsigned)(R.nparts * R.nch - 1));
    }
    __syncthreads();
    if (!last_cta) return;
    __threadfence();
    for (int c = 0; c < R.nch; ++c) {
        // eight independent chains hide the L2 latency; fixed combination order
        const double* pp = R.partials + (size_t)c * R.nparts;
        double a8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int i = tid;
        for (; i + 7 * nt < R.nparts; i += 8 * nt) {
#pragma unroll
            for (int k = 0; k < 8; ++k) a8[k] += __ldcg(pp + i + k * nt);
        }
        for (; i < R.nparts; i += nt) a8[0] += __ldcg(pp + i);
        double acc = ((a8[0] + a8[1]) + (a8[2] + a8[3])) + ((a8[4] + a8[5]) + (a8[6] + a8[7]));
        acc = block_sum_d(acc);
        if (tid == 0) R.out[c] = acc;
    }
    if (tid == 0) *R.ticket = 0u;
}

// Origin of subdomain b (side 32, stride s) along an axis of n pixels. The
// last subdomain is shifted back to end at the image border, so that every
// subdomain is a full 32 pixels whenever n >= 32 (same count and the same
// owned cores as the plain stride placement).
__host__ __device__ __forceinline__ int sub_origin_n(int b, int n, int s, int size) {
    if (n < size) return 0;
    const int o = b * s;
    return o > n - size ? n - size : o;
}
__host__ __device__ __forceinline__ int sub_origin(int b, int n, int s) { return sub_origin_n(b, n, s, 32); }

// Number of overlapping subdomains of side `size` with overlap `ov` along an
// axis of n pixels: ceil((n - ov) / (size - ov)), at least 1 (Sec. 3.3).
__host__ __device__ __forceinline__ int tile_count(int n, int size, int ov) {
    const int s = size - ov;
    const int c = (n - ov + s - 1) / s;
    return c < 1 ? 1 : c;
}

// ------------------------------------------------------ batched launches ---
//
// A batched launch runs one solver phase over many (image, channel) tasks of
// different sizes with a 1-D grid: task t owns the CTAs
// [cta0[t], cta0[t+1]) (prefix sums, cta0[ntasks] = grid size). Every CTA
// finds its task by binary search; a task's CTAs then behave exactly like the
// CTAs of a plain launch over that one image and channel.
__device__ __forceinline__ int find_task(const int* __restrict__ cta0, int ntasks, int block) {
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(cta0 + mid) <= block) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Segmented deterministic grid reduction of a batched launch: the CTAs of
// segment s deposit their partials at partials[base[s] + part], the last CTA
// of the whole launch sums every segment (one warp per segment, lane-strided
// partials in eight chains, fixed order) and writes *out[s]. Bitwise
// reproducible for a given task table.
struct SegReduce {
    double* partials;
    unsigned* ticket;          // zero before the launch; reset by the last CTA
    const int* base;           // [nseg + 1] partial offsets (base[nseg] = total partials)
    double* const* out;        // [nseg] destination of each segment's sum
    int nseg;
    int total_ctas;            // CTAs of the launch that commit
};

__device__ __forceinline__ void seg_reduce_commit(const SegReduce& R, int seg, int part, double block_total) {
    __shared__ bool last_cta;
    const int tid = linear_tid();
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    if (tid == 0) {
        R.partials[R.base[seg] + part] = block_total;
        __threadfence();
        const unsigned t = atomicAdd(R.ticket, 1u);
        last_cta = (t == (unsigned)(R.total_ctas - 1));
    }
    __syncthreads();
    if (!last_cta) return;
    __threadfence();
    const int lane = tid & 31, nw = nt >> 5;
    for (int s = tid >> 5; s < R.nseg; s += nw) {
        const int b0 = __ldcg(R.base + s), b1 = __ldcg(R.base + s + 1);
        double a8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int i = b0 + lane;
        for (; i + 7 * 32 < b1; i += 8 * 32) {
#pragma unroll
            for (int k = 0; k < 8; ++k) a8[k] += __ldcg(R.partials + i + k * 32);
        }
        for (; i < b1; i += 32) a8[0] += __ldcg(R.partials + i);
        double acc = ((a8[0] + a8[1]) + (a8[2] + a8[3])) + ((a8[4] + a8[5]) + (a8[6] + a8[7]));
        acc = warp_sum_d(acc);
        if (lane == 0) *R.out[s] = acc;
    }
    if (tid == 0) *R.ticket = 0u;
}

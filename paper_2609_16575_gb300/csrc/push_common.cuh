// Definitions shared by the particle kernels of the CIC tile step (push.cu) and of the
// quadratic-shape step (tsc.cu): the kernel arguments, the mover staging and a block
// reduction.
#pragma once
#include "pic_internal.cuh"

namespace gbpic {

__host__ __device__ constexpr size_t align128(size_t b) { return (b + 127) / 128 * 128; }
constexpr int MQ = 32;   // staged movers per warp (a particle step adds at most 32)

template <typename T> struct PushArgs {
    Geom g;
    ParticleArrays<T> pa;   // the block the step reads
    ParticleArrays<T> pb;   // the block the step writes (tile kernel, append)
    const int* hin;         // per tile: cell histogram of pa (TILE_CELLS ints)
    int* hout;              // per tile: cell histogram of pb, built by the step
    Fields<T> f;
    T eps;          // q dt / (2 m)
    T dtd[3];       // dt / d_d
    T cq[3];        // q / (dt d_p d_r) / jscale : fixed-point units per unit weight
    Rec<T>* movers;
    int mover_cap;
    Rec<T>* spill;
    int spill_cap;
    Counters* ctr;
    int parity;
    double* krec;   // optional: accumulate sum w m ((g_old + g_new)/2 - 1) here
    double mass;
    int xshift;     // 1: the window moves after this cycle (stored x cells drop by one)
    int wait_polls; // polls of the TMA staging wait before it gives up (ERRB_TIMEOUT); 0: at once
    // a tile split over several CTAs (grids with fewer tiles than SMs): `parts` CTAs per
    // tile, the tiles' output cell ranges (next free slot, TILE_CELLS per tile) and input
    // counts prepared by k_split_prep
    int parts;
    int* goff;
    int* cnt_in;
    // Esirkepov's deposit: the crossers' records, exported by the tile kernel's warps
    // (esk_wcap records per warp and tile, counts in esk_cnt) and deposited by
    // k_esk_crossers
    T* esk_buf;
    int* esk_cnt;
    int esk_wcap;
};

// Sum of one double per thread of the block, added to *dst by thread 0.
__device__ __forceinline__ void block_add_double(double v, double* dst) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ double red[PUSH_WARPS_MAX];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(dst, s);
    }
}

// Staged movers of one warp (mq records in shared memory) into the global mover list.
template <typename T>
__device__ __forceinline__ void movers_flush(const PushArgs<T>& A, const Rec<T>* sM, int& mq, int lane) {
    __syncwarp();
    int base = 0;
    if (lane == 0) base = atomicAdd(&A.ctr->mover_count[A.parity], mq);
    base = __shfl_sync(0xffffffffu, base, 0);
    bool over = false;
    for (int j = lane; j < mq; j += 32) {
        if (base + j < A.mover_cap) A.movers[base + j] = sM[j];
        else over = true;
    }
    if (over) atomicOr(&A.ctr->err, ERRB_OVERFLOW);
    __syncwarp();
    mq = 0;
}

// Output ranges of a tile step: exclusive scan of the input cell histogram hin (two
// cells per thread of the first 256 threads) into s_off, the output histogram s_hn
// cleared (or, with hn_from_input, set to the input histogram, for a step that then
// applies only the particles that change cell), the total into *s_total.  The caller
// synchronises the block before using them.
template <bool hn_from_input = false>
__device__ __forceinline__ void hist_scan(const int* hin, int* s_off, int* s_hn, int* s_wsum, int* s_total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool sc = threadIdx.x < 256;
    const int a0 = sc ? hin[2 * threadIdx.x] : 0, a1 = sc ? hin[2 * threadIdx.x + 1] : 0;
    int incl = a0 + a1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31 && sc) s_wsum[warp] = incl;
    __syncthreads();
    if (sc) {
        int woff = 0;
        for (int w2 = 0; w2 < warp; ++w2) woff += s_wsum[w2];
        const int excl = woff + incl - (a0 + a1);
        s_off[2 * threadIdx.x] = excl;
        s_off[2 * threadIdx.x + 1] = excl + a0;
        s_hn[2 * threadIdx.x] = hn_from_input ? a0 : 0;
        s_hn[2 * threadIdx.x + 1] = hn_from_input ? a1 : 0;
        if (threadIdx.x == 255) *s_total = woff + incl;
    }
}

// The quadratic-shape tile step (tsc.cu) for one species, launched by the CIC step's
// host code when the context's shape is PIC_SHAPE_TSC.
template <typename T> pic_status launch_tsc_push(pic_ctx* c, PushArgs<T>& A, bool ids, bool rec);
// The backward half step u^0 -> u^{-1/2} with the TSC gather (B^0 given).
template <typename T>
pic_status launch_tsc_backpush(pic_ctx* c, PushArgs<T>& A, const T* B0x, const T* B0y, const T* B0z);

}  // namespace gbpic

// Particle kernels of one PIC cycle (KEMPIC-3D, sections 2.4-2.5):
//   k_tile_push   one CTA per 8^3-cell tile: TMA-stages E, B of the tile and its
//                 guard cells into shared memory, gathers, Boris-pushes, moves and
//                 zigzag-deposits every particle of the tile into a shared fixed-point
//                 J tile, updates the stayers in their slots, writes movers to a list
//                 (leaving holes) and flushes J to HBM with integer atomics.
//   k_list_push   the same step for particles held in the spill list (global-memory
//                 gather and deposit).
//   k_inject      the moving window's new plasma, into the mover list.
//   k_append      puts movers into the segment of their new tile (or the spill list).
#include <cuda/std/cstdint>

#include "push_common.cuh"

namespace gbpic {

template <typename T> __host__ __device__ constexpr int box_elems() { return SB * SB * Prec<T>::BX; }
template <typename T> __host__ __device__ constexpr int box_stride() {
    // each staged box starts on a 128-byte boundary
    return ((box_elems<T>() * (int)sizeof(T) + 127) / 128) * 128 / (int)sizeof(T);
}
constexpr int JT_ELEMS = 3 * SJ3;   // elements of the shared J tile (8 bytes each: see tile_add)
constexpr int QCAP_ = 32;   // record queue per warp (QCAP below)
constexpr int PSX = 10, PSY = 10, PSZ = 9;   // z-paired staged fields: x, y -1..8, pair base z -1..7
constexpr int PS = PSX * PSY * PSZ;          // pairs per component
// Shared memory of the tile kernel, in order: the warps' record queues; the z-paired
// fields; the J tile, which first receives the six raw E, B boxes from TMA (it is
// cleared once they have been converted to pairs); the warps' staged movers; the
// mbarrier.  Offsets are
// multiples of 128 bytes.
constexpr int QWORDS_ = (QCAP_ * 14 > 32 * 14 + 16 ? QCAP_ * 14 : 32 * 14 + 16);   // QWORDS below
template <typename T> __host__ __device__ constexpr size_t region_a_bytes() {
    return align128((size_t)(Prec<T>::THREADS / 32) * QWORDS_ * sizeof(T));
}
template <typename T> __host__ __device__ constexpr size_t pairs_bytes() { return align128((size_t)6 * PS * 2 * sizeof(T)); }
template <typename T> __host__ __device__ constexpr size_t jtile_bytes() {
    return align128((size_t)JT_ELEMS * 8 > (size_t)6 * box_stride<T>() * sizeof(T) ? (size_t)JT_ELEMS * 8
                                                                                  : (size_t)6 * box_stride<T>() * sizeof(T));
}
template <typename T> __host__ __device__ constexpr size_t movers_bytes() {
    return align128((size_t)(Prec<T>::THREADS / 32) * MQ * sizeof(Rec<T>));
}
template <typename T> constexpr size_t tile_smem_bytes() {
    // + 128: the kernel rounds the dynamic shared base up to a 128-byte boundary
    return region_a_bytes<T>() + pairs_bytes<T>() + jtile_bytes<T>() + movers_bytes<T>() + 16 + 128;
}

// Index of the shared J tile element of (component, local x, y, z), -1..9 each.
__device__ __forceinline__ int tile_index(int comp, int x, int y, int z) {
    return comp * SJ3 + ((z + 1) * SJ + (y + 1)) * SJ + (x + 1);
}
// Offset of slot q (0..11, the order of segment_values) from the index of its cell's
// (component 0) origin edge.
__device__ __forceinline__ int slot_offset(int q) {
    int comp, ex, ey, ez;
    slot_edge(q, 0, 0, 0, comp, ex, ey, ez);
    return tile_index(comp, ex, ey, ez) - tile_index(0, 0, 0, 0);
}

// Warp-private record queue in shared memory for the few deposits that do not fit the
// per-lane sums (a particle starting outside its lane's cell, a cell crosser's second
// segment).  Queuing them and adding them later with 24 lanes (one record value per
// lane, two records per pass) keeps the warp converged instead of letting one lane
// run 12 atomics while the others idle.  Records are 13 words: 12 values, then the
// tile index of the cell's origin edge; a stride coprime to the 32 banks keeps the
// push and the drain free of bank conflicts.
constexpr int QCAP = QCAP_;   // records per warp: one record kind of a particle step adds at most
                              // 32 (the queue is drained before a kind that would not fit and
                              // before every flush); a flush stages 32
constexpr int QS = 14;        // words per record: 12 values, the key, one pad (pairs stay aligned)
// words of one warp's queue: QCAP records, or the 32 staged sums of a flush with the
// second half shifted by 16 words, whichever is larger
constexpr int QWORDS = (QCAP * QS > 32 * QS + 16 ? QCAP * QS : 32 * QS + 16);
static_assert(QWORDS == QWORDS_ && QS == 14, "queue layout of the shared-memory plan");
template <typename T> struct WarpQueue {
    T* rec;      // [QCAP][QS]
    __device__ __forceinline__ int& key(int j) const { return *reinterpret_cast<int*>(rec + j * QS + 12); }
    __device__ __forceinline__ void put(int j, int k, const typename Pair<T>::t v[6]) const {
        typename Pair<T>::t* r = reinterpret_cast<typename Pair<T>::t*>(rec + j * QS);
#pragma unroll
        for (int q = 0; q < 6; ++q) r[q] = v[q];
        key(j) = k;
    }
};

// Append, for every lane, the record (ka, va) if want_a and (kb, vb) if want_b: 12
// values of the cell with origin index k (warp-collective).  The queue is drained
// first whenever a kind's records would not fit; otherwise records accumulate until
// the row's flush, so one drain pass adds the records of several particle steps.  With
// Esirkepov's deposit the top of the queue's words holds the me stacked crosser
// records (esk_stack), which lowers the capacity; they are exported first when even
// an empty queue would not hold a kind's records.
template <typename T>
__device__ __forceinline__ void q_drain(WarpQueue<T> Q, int& qn, int lane, uint32_t sJa, int qoff);
// A warp's segment of the exported crosser records (Esirkepov's deposit): segment seg
// of buf, cap records each (every particle the warp can step), n of them written
// (warp-uniform).
template <typename T> struct EskOut {
    T* buf;
    int cap;
    int seg;
    int n;
};
template <typename T>
__device__ __forceinline__ void esk_flush(WarpQueue<T> Q, int& me, int lane, EskOut<T>& eo, Counters* ctr);
constexpr int ESK_WORDS = 10;   // X1[3], X2[3], cw[3], packed first node
constexpr int ESK_BATCH = 16;   // stacked crosser records per warp before they are processed
static_assert(32 * ESK_WORDS <= QWORDS, "one particle step's crosser records fit in the record queue");
__device__ __forceinline__ int q_cap(int me) {
    const int c = (QWORDS - me * ESK_WORDS) / QS;
    return c < QCAP ? c : QCAP;
}
template <typename T, bool ESK>
__device__ __forceinline__ void q_push(WarpQueue<T> Q, int& qn, int& me, EskOut<T>& eo, Counters* ctr, bool want_a,
                                       int ka, const typename Pair<T>::t va[6], bool want_b, int kb,
                                       const typename Pair<T>::t vb[6], int lane, uint32_t sJa, int qoff) {
    const unsigned ma = __ballot_sync(0xffffffffu, want_a), mb = ESK ? 0u : __ballot_sync(0xffffffffu, want_b);
    if (!(ma | mb)) return;
    const unsigned lt = (1u << lane) - 1u;
    if (qn + __popc(ma) > (ESK ? q_cap(me) : QCAP)) {
        q_drain(Q, qn, lane, sJa, qoff);
        if (ESK && __popc(ma) > q_cap(me)) esk_flush(Q, me, lane, eo, ctr);
    }
    if (want_a) Q.put(qn + __popc(ma & lt), ka, va);
    qn += __popc(ma);
    if (qn + __popc(mb) > (ESK ? q_cap(me) : QCAP)) {
        q_drain(Q, qn, lane, sJa, qoff);
        if (ESK && __popc(mb) > q_cap(me)) esk_flush(Q, me, lane, eo, ctr);
    }
    if (want_b) Q.put(qn + __popc(mb & lt), kb, vb);
    qn += __popc(mb);
}

// Add every queued record to the shared J tile: lane 12h + q (h = 0, 1) adds value q of
// records 2j + h; sJa is the tile's byte address, qoff this lane's slot offset.  The two
// records of a pass lie QS words apart: their 24 words fall in distinct banks.
template <typename T>
__device__ __forceinline__ void q_drain(WarpQueue<T> Q, int& qn, int lane, uint32_t sJa, int qoff) {
    __syncwarp();
    if (lane < 24) {
        const int h = lane >= 12 ? 1 : 0, q = lane - 12 * h;
        for (int j = h; j < qn; j += 2) tile_add(sJa, Q.key(j) + qoff, JT_ELEMS, Q.rec[j * QS + q]);
    }
    __syncwarp();
    qn = 0;
}

// Warp flush of per-lane current sums acc (12 edge values of the cell with origin
// index key, or none for key < 0) into the shared J tile.  The 32 sums are staged in
// the (empty) record queue (the second half 16 words further, so that the two halves'
// reads fall in distinct banks); then lane 12h + q walks records 16h .. 16h + 15 of
// value q and adds one sum per run of equal keys.  The segments being sorted by cell,
// the keys of a warp form a few runs, so a flush costs a few atomics per value instead
// of 32 (shared atomics from many lanes on one address serialise).  A run ends for all
// lanes of a half at once; the additions of both halves are issued together.
template <typename T>
__device__ __forceinline__ void flush_warp(const typename Pair<T>::t acc[6], int key, int lane, WarpQueue<T> Q,
                                           uint32_t sJa, int qoff) {
    WarpQueue<T> S;
    S.rec = Q.rec + (lane >= 16 ? 16 : 0);
    S.put(lane, key, acc);
    __syncwarp();
    if (lane < 24) {
        const int h = lane >= 12 ? 1 : 0, q = lane - 12 * h;
        WarpQueue<T> W;
        W.rec = Q.rec + 16 * h;
        int ck = -1;
        T sum = T(0);
#pragma unroll
        for (int j = 16 * h; j < 16 * h + 16; ++j) {
            const int k = W.key(j);
            const T v = W.rec[j * QS + q];
            const bool brk = k != ck;
            if (__any_sync(0x00ffffffu, brk)) {
                if (brk && ck >= 0 && sum != T(0)) tile_add(sJa, ck + qoff, JT_ELEMS, sum);
                if (brk) {
                    ck = k;
                    sum = T(0);
                }
            }
            sum += v;
        }
        if (ck >= 0 && sum != T(0)) tile_add(sJa, ck + qoff, JT_ELEMS, sum);
    }
    __syncwarp();
}

// Gather E and B (section 2.5) from the tile's z-paired staged fields sP: pair
// (F(x, y, z), F(x, y, z + 1)) of component c at local (x, y, z) is
// sP[c PS + ((z + 1) PSY + (y + 1)) PSX + x + 1].  The cell's pair index is
// computed once and each component's stencil origin is a fixed offset from it (a
// half-located dimension shifts by -1 when the offset is below one half).  Each
// component is the trilinear interpolation of trilerp (x, then y, then z), with the
// x and y stages done on both z planes at once.
template <typename T>
__device__ __forceinline__ void gather_tile(const typename Pair<T>::t* sP, int x, int y, int z, T dx, T dy, T dz,
                                            T Ep[3], T Bp[3]) {
    using PT = Pair<T>;
    using P2 = typename PT::t;
    const bool ux = dx >= T(0.5), uy = dy >= T(0.5), uz = dz >= T(0.5);
    const T shx = ux ? dx - T(0.5) : dx + T(0.5);
    const T shy = uy ? dy - T(0.5) : dy + T(0.5);
    const T shz = uz ? dz - T(0.5) : dz + T(0.5);
    const int ox = ux ? 0 : -1, oy = uy ? 0 : -PSX, oz = uz ? 0 : -PSX * PSY;
    const P2* p = sP + ((z + 1) * PSY + (y + 1)) * PSX + (x + 1);
    auto tri = [&](const P2* q, T sx, T sy, T sz) -> T {
        const P2 a00 = q[0], a10 = q[1], a01 = q[PSX], a11 = q[PSX + 1];
        const P2 sx2 = PT::splat(sx);
        const P2 q0 = PT::fma(sx2, PT::sub(a10, a00), a00);
        const P2 q1 = PT::fma(sx2, PT::sub(a11, a01), a01);
        const P2 r = PT::fma(PT::splat(sy), PT::sub(q1, q0), q0);
        return r.x + sz * (r.y - r.x);
    };
    // E: Ex (h,n,n), Ey (n,h,n), Ez (n,n,h);  B: Bx (n,h,h), By (h,n,h), Bz (h,h,n)
    Ep[0] = tri(p + 0 * PS + ox, shx, dy, dz);
    Ep[1] = tri(p + 1 * PS + oy, dx, shy, dz);
    Ep[2] = tri(p + 2 * PS + oz, dx, dy, shz);
    Bp[0] = tri(p + 3 * PS + oy + oz, dx, shy, shz);
    Bp[1] = tri(p + 4 * PS + ox + oz, shx, dy, shz);
    Bp[2] = tri(p + 5 * PS + ox + oy, shx, shy, dz);
}

// Cells of a lane's R slots (one 16- or 8-byte load) and the start cell its current
// sums are kept for: the cell most of the R particles start in (a particle that crossed
// a cell face last step, or a cell boundary inside the group, then costs one queued
// record instead of R - 1).
template <int R> struct RowCells;
template <> struct RowCells<4> {
    static __device__ __forceinline__ void ld(const int* p, int c[4]) {
        const int4 a = __ldg(reinterpret_cast<const int4*>(p));
        c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
    }
    static __device__ __forceinline__ void st(int* p, const int c[4]) {
        __stcs(reinterpret_cast<int4*>(p), make_int4(c[0], c[1], c[2], c[3]));
    }
    static __device__ __forceinline__ int key(const int c[4]) {
        int k = c[2] == c[3] ? c[2] : c[1];
        if (k < 0) k = c[0] >= 0 ? c[0] : (c[1] >= 0 ? c[1] : (c[2] >= 0 ? c[2] : c[3]));
        return k;
    }
};
template <> struct RowCells<2> {
    static __device__ __forceinline__ void ld(const int* p, int c[2]) {
        const int2 a = __ldg(reinterpret_cast<const int2*>(p));
        c[0] = a.x; c[1] = a.y;
    }
    static __device__ __forceinline__ void st(int* p, const int c[2]) {
        __stcs(reinterpret_cast<int2*>(p), make_int2(c[0], c[1]));
    }
    static __device__ __forceinline__ int key(const int c[2]) { return c[0] >= 0 ? c[0] : c[1]; }
};

// Esirkepov's deposit of the cell crossers.  A crosser's record (positions relative to
// the first node of its support, cw, the first node and the crossed dimensions packed)
// is stacked at the top of the warp's record-queue words, record e at
// QWORDS - (e + 1) ESK_WORDS, beside the ZigZag-style records below, so that a crosser
// does not force the record queue to drain; a batch of up to ESK_BATCH records is
// copied at once to the warp's segment of the global record list, and k_esk_crossers
// deposits the list after the tile kernel.  (Deposited inside the tile kernel, with the
// batch's values spread over the lanes, the crossers had cost the kernel a third of its
// time: the deposit ran at the kernel's low issue rate and its code crowded the
// instruction cache.)
template <typename T> __device__ __forceinline__ T* esk_rec(WarpQueue<T> Q, int e) {
    return Q.rec + QWORDS - (e + 1) * ESK_WORDS;
}
// The stacked batch out of the queue words into the warp's export segment (the records
// e = me - 1 .. 0 are contiguous words).  The segment holds every particle the warp can
// step, so it cannot fill; a batch that would not fit (a broken launch) is dropped with
// the overflow error bit.
template <typename T>
__device__ __forceinline__ void esk_flush(WarpQueue<T> Q, int& me, int lane, EskOut<T>& eo, Counters* ctr) {
    __syncwarp();
    if (eo.n + me <= eo.cap) {
        const T* src = esk_rec(Q, me - 1);
        T* dst = eo.buf + ((size_t)eo.seg * eo.cap + eo.n) * ESK_WORDS;
        for (int j = lane; j < me * ESK_WORDS; j += 32) dst[j] = src[j];
        eo.n += me;
    } else if (lane == 0) {
        atomicOr(&ctr->err, ERRB_OVERFLOW);
    }
    __syncwarp();
    me = 0;
}

// Esirkepov's deposit of one exported crosser record into a shared J tile (one thread):
// its non-zero values (along a dimension the move did not cross, the third node and the
// second edge carry nothing: 20 of the 3x3x3 support's 54 for a move across one face),
// in esk_value's arithmetic, with the node weights S0 and DS = S1 - S0 of each dimension
// computed once for the record.
template <typename T>
__device__ __forceinline__ void esk_record(const T* rec, uint32_t sJa) {
    const T X1[3] = {rec[0], rec[1], rec[2]}, X2[3] = {rec[3], rec[4], rec[5]};
    const int pk = *reinterpret_cast<const int*>(rec + 9);
    const int base = tile_index(0, (pk & 15) - 1, ((pk >> 4) & 15) - 1, ((pk >> 8) & 15) - 1);
    const int crossed[3] = {(pk >> 12) & 1, (pk >> 13) & 1, (pk >> 14) & 1};
    T s0[3][3], ds[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            s0[k][j] = cic_w(X1[k] - T(j));
            ds[k][j] = cic_w(X2[k] - T(j)) - s0[k][j];
        }
    constexpr int stride[3] = {1, SJ, SJ * SJ};
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
        const int p = comp == 2 ? 0 : comp + 1, r = comp == 0 ? 2 : comp - 1;
        const T cw = rec[6 + comp];
        const int e0 = base + comp * SJ3;
#pragma unroll
        for (int jp = 0; jp < 3; ++jp) {
            if (jp == 2 && !crossed[p]) continue;
#pragma unroll
            for (int jr = 0; jr < 3; ++jr) {
                if (jr == 2 && !crossed[r]) continue;
                const T t = s0[p][jp] * s0[r][jr] + T(0.5) * ds[p][jp] * s0[r][jr] + T(0.5) * s0[p][jp] * ds[r][jr] +
                            ds[p][jp] * ds[r][jr] * T(1.0 / 3.0);
                const int e = e0 + jp * stride[p] + jr * stride[r];
                T acc = ds[comp][0] * t;
                const T v0 = -cw * acc;
                if (v0 != T(0)) tile_add(sJa, e, JT_ELEMS, v0);
                if (crossed[comp]) {
                    acc += ds[comp][1] * t;
                    const T v1 = -cw * acc;
                    if (v1 != T(0)) tile_add(sJa, e + stride[comp], JT_ELEMS, v1);
                }
            }
        }
    }
}

// Stack the records of this particle step's crossers (mine), exporting the stacked
// batch first when it would grow past ESK_BATCH or meet the queued records.
template <typename T>
__device__ __forceinline__ void esk_stack(WarpQueue<T> Q, int& qn, int& me, EskOut<T>& eo, Counters* ctr, int lane,
                                          uint32_t sJa, int qoff, bool mine, int x, int y, int z, const T d1[3], const T d2[3],
                                          const int s[3], const T cw[3]) {
    const unsigned mc = __ballot_sync(0xffffffffu, mine);
    const int nn = __popc(mc);
    if (me + nn > ESK_BATCH || qn * QS + (me + nn) * ESK_WORDS > QWORDS) esk_flush(Q, me, lane, eo, ctr);
    if (qn * QS + (me + nn) * ESK_WORDS > QWORDS) q_drain(Q, qn, lane, sJa, qoff);
    if (mine) {
        T* rec = esk_rec(Q, me + __popc(mc & ((1u << lane) - 1u)));
        int b[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            b[k] = s[k] < 0 ? -1 : 0;
            rec[k] = d1[k] - T(b[k]);
            rec[3 + k] = d2[k] + T(s[k] - b[k]);
            rec[6 + k] = cw[k];
        }
        // first node of the support (local -1 .. 7 per dimension, 4 bits each) and which
        // dimensions the move crossed (one bit each)
        *reinterpret_cast<int*>(rec + 9) = (x + b[0] + 1) | ((y + b[1] + 1) << 4) | ((z + b[2] + 1) << 8) |
                                           ((s[0] != 0) << 12) | ((s[1] != 0) << 13) | ((s[2] != 0) << 14);
    }
    me += nn;
}

// Write a warp's mq staged movers to the global mover list: one counter atomic per
// batch (the only global atomic whose result a warp waits for), then the records by
// the lanes (warp-collective).
// Start of a tile: one thread issues the six TMA box loads of E and B
// (local cells -1..8, origin at the tile's ghost corner) completing on one mbarrier while
// the first 256 threads scan the input cell histogram into the output cell ranges; then
// the boxes are rewritten as z pairs and the J tile that shared their space is cleared.
// The wait for the boxes is bounded by A.wait_polls polls: a tile that gives up raises
// ERRB_TIMEOUT, waits (bounded again, MBAR_MAX_POLLS) for the copies in flight, drops its
// particles (count, holes and the output histogram set to zero, so later steps read
// nothing stale) and returns false.
template <typename T, int NT, bool SCAN = true>
__device__ __forceinline__ bool tile_prologue(const PushArgs<T>& A, int tile, int cnt, int ox, int oy, int oz,
                                              const int* hin, int* hout, const CUtensorMap& tE0,
                                              const CUtensorMap& tE1, const CUtensorMap& tE2,
                                              const CUtensorMap& tB0, const CUtensorMap& tB1,
                                              const CUtensorMap& tB2, T* sF, typename Pair<T>::t* sP,
                                              unsigned char* sJ, uint64_t* bar, int* s_off, int* s_hn, int* s_wsum,
                                              int* s_timeout, int* s_total, int* s_left) {
    constexpr int BX = Prec<T>::BX;
    constexpr int BS = box_stride<T>();
    static_assert(NT >= 256 && NT % 32 == 0, "the histogram scan uses the first 256 threads");
    if (threadIdx.x == 0) {
        *s_timeout = 0;
        *s_left = 0;
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(bar, 6u * box_elems<T>() * sizeof(T));
        // padded coordinate of local cell -1 is the tile origin itself
        tma_load_3d(sF + 0 * BS, &tE0, ox, oy, oz, bar);
        tma_load_3d(sF + 1 * BS, &tE1, ox, oy, oz, bar);
        tma_load_3d(sF + 2 * BS, &tE2, ox, oy, oz, bar);
        tma_load_3d(sF + 3 * BS, &tB0, ox, oy, oz, bar);
        tma_load_3d(sF + 4 * BS, &tB1, ox, oy, oz, bar);
        tma_load_3d(sF + 5 * BS, &tB2, ox, oy, oz, bar);
    }
    // output ranges: exclusive scan of the input histogram (a split tile's ranges come
    // from k_split_prep)
    if (SCAN) hist_scan<true>(hin, s_off, s_hn, s_wsum, s_total);
    for (int polls = 0;; ++polls) {
        if (polls >= A.wait_polls) {   // (a bound of 0 gives up without waiting)
            *s_timeout = 1;
            break;
        }
        if (mbar_try_wait(bar, 0)) break;
    }
    __syncthreads();
    if (*s_timeout) {
        if (threadIdx.x == 0) {
            atomicOr(&A.ctr->err, ERRB_TIMEOUT);
            // wait (bounded) for the copies still in flight before the CTA exits
            int polls = 0;
            while (!mbar_try_wait(bar, 0) && ++polls < MBAR_MAX_POLLS) {
            }
            A.pa.count[tile] = 0;
            A.pa.holes[tile] = 0;
        }
        for (int i = threadIdx.x; i < TILE_CELLS; i += NT) hout[i] = 0;
        __syncthreads();
        return false;
    }
    // z pairs (F(x, y, z), F(x, y, z + 1)) of every component, local x, y -1..8, z -1..7:
    // one x row of PSX pairs per thread and pass
    for (int row = threadIdx.x; row < 6 * PSZ * PSY; row += NT) {
        const int c = row / (PSZ * PSY), r = row - c * (PSZ * PSY);
        const int zi = r / PSY, yi = r - zi * PSY;
        const T* F = sF + c * BS + (zi * SB + yi) * BX;
        typename Pair<T>::t* dst = sP + c * PS + (zi * PSY + yi) * PSX;
#pragma unroll
        for (int xi = 0; xi < PSX; ++xi) dst[xi] = Pair<T>::make(F[xi], F[xi + SB * BX]);
    }
    __syncthreads();   // the raw boxes are consumed: clear the J tile in their place
    {
        unsigned long long* z = reinterpret_cast<unsigned long long*>(sJ);
        for (int i = threadIdx.x; i < JT_ELEMS; i += NT) z[i] = 0ull;
    }
    __syncthreads();
    return true;
}

// The J tile into HBM: element (comp, lx, ly, lz), local -1..9, is
// added to the global edge of its wrapped cell (the periodic guard layers fold onto the
// other side of the box; what lies outside an open x is dropped) with the 64-bit
// fixed-point (FP32) or FP64 atomic add.  gidx[SJ d + l + 1] is the global index along
// dimension d of local l (x: -1 outside an open x), filled by the caller.
template <typename T, int NT>
__device__ __forceinline__ void tile_flush_j(const PushArgs<T>& A, const unsigned char* sJ, const int* gidx) {
    using Acc = typename JTraits<T>::acc_t;
    for (int e = threadIdx.x; e < JT_ELEMS; e += NT) {
        const Acc v = tile_get(sJ, e, JT_ELEMS, T(0));
        if (v == Acc(0)) continue;
        const int comp = e / SJ3, r = e - comp * SJ3;
        const int lz = r / (SJ * SJ), r2 = r - lz * (SJ * SJ);
        const int ly = r2 / SJ, lx = r2 - ly * SJ;
        const int gx = gidx[lx];
        if (gx < 0) continue;   // current leaving an open x face
        acc_atomic(A.f.J[comp] + A.g.cidx(gx, gidx[SJ + ly], gidx[2 * SJ + lz]), v);
    }
}
// Fill the table of tile_flush_j (threads 0 .. 3 SJ - 1).
template <typename T>
__device__ __forceinline__ void tile_flush_index(const PushArgs<T>& A, int ox, int oy, int oz, int* gidx) {
    const int t = threadIdx.x;
    if (t < 3 * SJ) {
        const int d = t / SJ, l = t - d * SJ - 1;
        gidx[t] = d == 0 ? x_after(A.g, ox + l) : (d == 1 ? wrap_idx(oy + l, A.g.n[1]) : wrap_idx(oz + l, A.g.n[2]));
    }
}

// One CTA per tile.  The tile's particles are read from one SoA block and written to
// the other, grouped by the cell each particle starts the step in: the block read is
// grouped by the cells of the step before, so only the particles that crossed a cell
// face last step (and the movers appended at the segment's end) are out of place.  The
// output ranges come from the cell histogram of the input (kept from the previous
// step); a particle that leaves the tile leaves a hole in its range, and the histogram
// of the output's cells is built for the next step.  Lane l of warp w handles the R
// consecutive input slots of slot group 32 row + l for rows w, w + warps, ...; a lane's
// R particles nearly always start in one cell: their straight-segment currents are
// summed in registers and each row ends with one warp flush of those sums; everything
// else goes through the warp's record queue.
template <typename T, bool IDS, bool RECK, bool ESK, bool SPLIT>
__global__ void __launch_bounds__(Prec<T>::THREADS, Prec<T>::MINB)
k_tile_push(const __grid_constant__ CUtensorMap tE0, const __grid_constant__ CUtensorMap tE1,
            const __grid_constant__ CUtensorMap tE2, const __grid_constant__ CUtensorMap tB0,
            const __grid_constant__ CUtensorMap tB1, const __grid_constant__ CUtensorMap tB2, PushArgs<T> A) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    using Acc = typename JTraits<T>::acc_t;
    constexpr int NT = Prec<T>::THREADS, NW = NT / 32, R = Prec<T>::R;
    static_assert(NW <= PUSH_WARPS_MAX, "tile kernel CTA too large");
    using P2 = typename Pair<T>::t;
    unsigned char* sQ = smem;
    P2* sP = reinterpret_cast<P2*>(smem + region_a_bytes<T>());
    unsigned char* sJ = smem + region_a_bytes<T>() + pairs_bytes<T>();
    T* sF = reinterpret_cast<T*>(sJ);                       // raw boxes, then the J tile
    const uint32_t sJa = smem_u32(sJ);
    Rec<T>* sM = reinterpret_cast<Rec<T>*>(sJ + jtile_bytes<T>()) + (threadIdx.x >> 5) * MQ;   // this warp's movers
    uint64_t* bar = reinterpret_cast<uint64_t*>(sJ + jtile_bytes<T>() + movers_bytes<T>());
    __shared__ int s_off[TILE_CELLS];   // next free output slot of each input cell's range
    __shared__ int s_hn[TILE_CELLS];    // cell histogram of the output
    __shared__ int s_wsum[8];
    __shared__ int s_timeout, s_total, s_left;

    // a split tile is handled by A.parts CTAs, part p taking every A.parts-th row of
    // each warp's rows; its output ranges and histogram then live in global memory
    const int tile = SPLIT ? blockIdx.x / A.parts : blockIdx.x;
    const int part = SPLIT ? blockIdx.x - tile * A.parts : 0;
    const int nparts = SPLIT ? A.parts : 1;
    const int cnt = min(SPLIT ? A.cnt_in[tile] : A.pa.count[tile], A.pa.cap[tile]);
    const int* hin = A.hin + (size_t)tile * TILE_CELLS;
    int* hout = A.hout + (size_t)tile * TILE_CELLS;
    int* const offp = SPLIT ? A.goff + (size_t)tile * TILE_CELLS : s_off;   // next free output slot per cell
    int* const hnp = SPLIT ? hout : s_hn;                                 // output histogram
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (cnt == 0) {
        if (!SPLIT) {
            for (int i = threadIdx.x; i < TILE_CELLS; i += NT) hout[i] = 0;
            if (threadIdx.x == 0) A.pa.holes[tile] = 0;
        }
        return;
    }
    const int ntx = A.g.nt[0], nty = A.g.nt[1];
    const int tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
    const int ox = tx * TILE, oy = ty * TILE, oz = tz * TILE;

    if (!tile_prologue<T, NT, !SPLIT>(A, tile, cnt, ox, oy, oz, hin, hout, tE0, tE1, tE2, tB0, tB1, tB2, sF, sP, sJ,
                                       bar, s_off, s_hn, s_wsum, &s_timeout, &s_total, &s_left))
        return;

    const int ext[3] = {min(TILE, A.g.n[0] - ox), min(TILE, A.g.n[1] - oy), min(TILE, A.g.n[2] - oz)};
    WarpQueue<T> Q;
    Q.rec = reinterpret_cast<T*>(sQ) + (size_t)warp * QWORDS;
    const int qoff = slot_offset(lane < 12 ? lane : (lane < 24 ? lane - 12 : 0));
    int qn = 0;                   // queued records (warp-uniform)
    int me = 0;                   // stacked Esirkepov crosser records (warp-uniform)
    EskOut<T> eo{A.esk_buf, A.esk_wcap, tile * NW + warp, 0};   // this warp's export segment
    const int seg = A.pa.seg_start[tile];   // slots of a block are below 2^31
    const int ngroups = (cnt + R - 1) / R;
    double kacc = 0.0;
    int left = 0;                 // particles this lane moved out of the tile or removed
    int esc = 0;                  // of those, removed at an open x face
    int mq = 0;                   // staged movers of this warp (warp-uniform)
    // the next particle's state, loaded one particle step ahead (cached in L2 only: with
    // shared memory taking most of the SM, L1 kept few of the sectors that the R slots of
    // a lane share, and bypassing it measured 1 % faster)
    int n_lc = HOLE;
    T n_d[3], n_u[3], n_w;
    auto prefetch = [&](int i) {
        const bool in = i < cnt;
        const int q = seg + (in ? i : 0);   // slots past count read slot 0, unused
        const int c = __ldcg(A.pa.cell + q);
        n_lc = in ? c : HOLE;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            n_d[k] = __ldcg(A.pa.d[k] + q);
            n_u[k] = __ldcg(A.pa.u[k] + q);
        }
        n_w = __ldcg(A.pa.w + q);
    };
    const int row0 = warp + NW * part, rstep = NW * nparts;   // this warp's rows
    prefetch((row0 * 32 + lane) * R);
    int n_cells[R];               // the cells of the next row's R slots
    auto prefetch_cells = [&](int i0) {
        if (i0 < cnt) RowCells<R>::ld(A.pa.cell + seg + i0, n_cells);
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (i0 + r >= cnt) n_cells[r] = HOLE;
    };
    prefetch_cells((row0 * 32 + lane) * R);

    for (int row = row0; row * 32 < ngroups; row += rstep) {
        P2 acc[6];                // summed straight-segment currents of start cell `key`
        int key = RowCells<R>::key(n_cells);
        // output slots: the lanes whose R particles start in one cell claim R slots each
        // of that cell's range with one shared atomic per warp and cell; the other lanes
        // claim one slot per particle below
        bool uni = n_cells[0] >= 0;
#pragma unroll
        for (int r = 1; r < R; ++r) uni = uni && n_cells[r] == n_cells[0];
        int obase, ostride;
        {
            const unsigned grp = __match_any_sync(0xffffffffu, uni ? n_cells[0] : -1 - lane);
            const int leader = __ffs(grp) - 1;
            int b = 0;
            if (uni && lane == leader) b = atomicAdd(&offp[n_cells[0]], R * __popc(grp));
            b = __shfl_sync(0xffffffffu, b, leader);
            // particle r of the group's k-th lane takes slot b + r G + k (G lanes): at each
            // particle step the group writes G consecutive slots
            obase = uni ? b + __popc(grp & ((1u << lane) - 1u)) : -1;
            ostride = __popc(grp);
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) acc[q] = Pair<T>::splat(T(0));
        const int s0 = (row * 32 + lane) * R;   // first slot of this lane
        prefetch_cells(((row + rstep) * 32 + lane) * R);
#pragma unroll 1
        for (int r = 0; r < R; ++r) {
            const int i = s0 + r;
            const int p = seg + i;
            const int lc = n_lc;
            const bool active = lc >= 0;
            T u[3] = {n_u[0], n_u[1], n_u[2]}, d2[3] = {T(0), T(0), T(0)}, w = n_w;
            const T d1[3] = {n_d[0], n_d[1], n_d[2]};
            prefetch(r + 1 < R ? i + 1 : ((row + rstep) * 32 + lane) * R);
            P2 v[6], v2[6];
            T cw[3] = {T(0), T(0), T(0)};
            int s[3] = {0, 0, 0};
            int x = 0, y = 0, z = 0, nlc = -1;
            bool stay = false, move = false, crossed = false;
            if (active) {
                x = lc & 7;
                y = (lc >> 3) & 7;
                z = lc >> 6;
                T Ep[3], Bp[3];
                gather_tile<T>(sP, x, y, z, d1[0], d1[1], d1[2], Ep, Bp);
                T gm1_old = T(0);
                if (RECK) gm1_old = gamma_minus_one(u);
                const T ig = boris(A.eps, Ep, Bp, u);
                if (RECK) kacc += (double)w * A.mass * 0.5 * ((double)gm1_old + (double)gamma_minus_one(u));
                bool far = false;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    s[k] = advance(d1[k], A.dtd[k] * u[k] * ig, d2[k]);
                    far = far || s[k] > 1 || s[k] < -1;
                    s[k] = max(-1, min(1, s[k]));
                }
                const int errb = (ig > T(0) ? 0 : ERRB_NAN) | (far ? ERRB_SUPERLUMINAL : 0);
                if (errb) atomicOr(&A.ctr->err, errb);
#pragma unroll
                for (int k = 0; k < 3; ++k) cw[k] = A.cq[k] * w;
                crossed = (s[0] | s[1] | s[2]) != 0;
                // the segment in the start cell, without a branch: for a particle that
                // stays in its cell both zigzag segments lie there, and their two
                // midpoint products and D_p D_r / 48 terms add up to the straight
                // segment x1 -> x2 (midpoint weights, D_p D_r / 12 term); for a crosser
                // it is the relay split's first segment.  The second segment's flux and
                // midpoint follow below, once for the warp's crossers.
                const T h = crossed ? T(0.5) : T(1);
                T Fa[3], Wa[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const T D = d2[k] - d1[k];
                    const T up = s[k] > 0 ? T(1) : T(0);
                    Fa[k] = s[k] == 0 ? h * D : up - d1[k];
                    Wa[k] = s[k] == 0 ? d1[k] + T(0.5) * h * D : T(0.5) * (d1[k] + up);
                }
                segment_values_pairs(cw, Fa, Wa, v);
                // when the window moves after this cycle the stored x cell drops by one; a
                // particle that crossed the window's front face leaves all the same
                const int nx = x + s[0] - A.xshift, ny = y + s[1], nz = z + s[2];
                stay = nx >= 0 && nx < ext[0] && ny >= 0 && ny < ext[1] && nz >= 0 && nz < ext[2] &&
                       (A.xshift == 0 || ox + x + s[0] < A.g.n[0]);
                move = !stay;
                if (stay) nlc = nx | (ny << 3) | (nz << 6);
                // the particle's slot in its start cell's output range: the state after
                // the step, or a hole
                const int o = seg + (obase >= 0 ? obase + r * ostride : atomicAdd(&offp[lc], 1));
                __stcs(A.pb.cell + o, stay ? nlc : HOLE);
                if (stay) {
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        __stcs(A.pb.d[k] + o, d2[k]);
                        __stcs(A.pb.u[k] + o, u[k]);
                    }
                    __stcs(A.pb.w + o, w);
                    if (IDS) __stcs(A.pb.id + o, __ldg(A.pa.id + p));
                } else {
                    ++left;
                }
            }
            // cell histogram of the output: it starts as the input histogram (every
            // particle counted in its start cell); a particle that changes cell or leaves
            // the tile moves its count.  In a cycle that ends with a window move every
            // stored cell changes: the counts then move once per warp and cell.
            if (A.xshift == 0) {
                if (active && nlc != lc) {
                    atomicSub(&hnp[lc], 1);
                    if (nlc >= 0) atomicAdd(&hnp[nlc], 1);
                }
            } else {
                const unsigned g1 = __match_any_sync(0xffffffffu, active ? lc : -1 - lane);
                if (active && lane == __ffs(g1) - 1) atomicSub(&hnp[lc], __popc(g1));
                const unsigned g2 = __match_any_sync(0xffffffffu, nlc >= 0 ? nlc : -1 - lane);
                if (nlc >= 0 && lane == __ffs(g2) - 1) atomicAdd(&hnp[nlc], __popc(g2));
            }
            // a crosser's second segment, in the cell it moved to (relay split)
            if (!ESK && __any_sync(0xffffffffu, crossed)) {
                T F2[3], W2[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const T dn = s[k] < 0 ? T(1) : T(0);
                    F2[k] = s[k] == 0 ? T(0.5) * (d2[k] - d1[k]) : d2[k] - dn;
                    W2[k] = s[k] == 0 ? d1[k] + T(0.75) * (d2[k] - d1[k]) : T(0.5) * (d2[k] + dn);
                }
                segment_values_pairs(cw, F2, W2, v2);
            }
            // with Esirkepov's deposit a crosser's whole current is its own stencil (below)
            const bool esk_cross = ESK && crossed;
            const bool summed = active && lc == key && !esk_cross;
            if (summed) {
#pragma unroll
                for (int q = 0; q < 6; ++q) acc[q] = Pair<T>::add(acc[q], v[q]);
            }
            q_push<T, ESK>(Q, qn, me, eo, A.ctr, active && !summed && !esk_cross, tile_index(0, x, y, z), v, !ESK && crossed,
                           tile_index(0, x + s[0], y + s[1], z + s[2]), v2, lane, sJa, qoff);
            if (ESK && __any_sync(0xffffffffu, esk_cross))
                esk_stack<T>(Q, qn, me, eo, A.ctr, lane, sJa, qoff, esk_cross, x, y, z, d1, d2, s, cw);
            // movers: staged in shared memory with their wrapped global cell and written to
            // the global list in batches; a particle that left an open x face is removed
            // instead
            int gxm = 0;
            if (move) {
                gxm = x_after1(A.g, ox + x + s[0]);
                if (gxm >= 0) gxm -= A.xshift;   // the window's first column leaves
                if (gxm < 0) {
                    move = false;
                    ++esc;
                }
            }
            if (const unsigned mm = __ballot_sync(0xffffffffu, move)) {
                if (mq + __popc(mm) > MQ) movers_flush(A, sM, mq, lane);
                if (move) {
                    Rec<T>& rc = sM[mq + __popc(mm & ((1u << lane) - 1u))];
                    const int gy = wrap1(oy + y + s[1], A.g.n[1]);
                    const int gz = wrap1(oz + z + s[2], A.g.n[2]);
                    rc.cell = (gz * A.g.n[1] + gy) * A.g.n[0] + gxm;
                    rc.id = IDS ? A.pa.id[p] : 0;
                    rc.d[0] = d2[0];
                    rc.d[1] = d2[1];
                    rc.d[2] = d2[2];
                    rc.u[0] = u[0];
                    rc.u[1] = u[1];
                    rc.u[2] = u[2];
                    rc.w = w;
                }
                mq += __popc(mm);
            }
        }
        if (qn) q_drain(Q, qn, lane, sJa, qoff);   // the flush stages its sums in the queue
        if (ESK && me) esk_flush(Q, me, lane, eo, A.ctr);
        flush_warp<T>(acc, key >= 0 ? tile_index(0, key & 7, (key >> 3) & 7, key >> 6) : -1, lane, Q, sJa, qoff);
    }
    if (mq) movers_flush(A, sM, mq, lane);
    if (ESK && lane == 0) A.esk_cnt[(size_t)tile * NW + warp] = eo.n;
    left = __reduce_add_sync(0xffffffffu, left);
    esc = __reduce_add_sync(0xffffffffu, esc);
    if (lane == 0 && left) atomicAdd(SPLIT ? &A.pa.holes[tile] : &s_left, left);
    if (lane == 0 && esc) atomicAdd(&A.ctr->escaped, esc);
    __shared__ int s_gidx[3 * SJ];
    tile_flush_index(A, ox, oy, oz, s_gidx);
    __syncthreads();
    // the output segment: the input cells' ranges (with the holes of the departed) and,
    // appended later, this step's arrivals (a split tile's count, holes and histogram are
    // set by k_split_prep and updated in global memory)
    if (!SPLIT) {
        for (int i = threadIdx.x; i < TILE_CELLS; i += NT) hout[i] = s_hn[i];
        if (threadIdx.x == 0) {
            A.pa.count[tile] = s_total;
            A.pa.holes[tile] = s_left;
        }
    }
    // flush the shared J tile to HBM (periodic wrap of the guard layers)
    tile_flush_j<T, NT>(A, sJ, s_gidx);
    if (RECK) block_add_double(kacc, A.krec);
}

// Esirkepov's deposit of the crossers a tile kernel exported: one CTA per tile, one
// record per thread into a shared J tile of the tile kernel's layout, then the tile's
// flush into HBM.  The counts it consumed are zeroed for the next step (a tile kernel
// CTA that leaves early, on an empty tile or a staging timeout, writes no counts).
template <typename T>
__global__ void __launch_bounds__(256) k_esk_crossers(PushArgs<T> A) {
    constexpr int NW = Prec<T>::THREADS / 32;
    extern __shared__ __align__(16) unsigned char sJc[];
    __shared__ int s_pre[NW + 1];
    __shared__ int s_gidx[3 * SJ];
    const int tile = blockIdx.x;
    int* cnt = A.esk_cnt + (size_t)tile * NW;
    if (threadIdx.x == 0) {
        int sum = 0;
        for (int w = 0; w < NW; ++w) {
            s_pre[w] = sum;
            sum += min(cnt[w], A.esk_wcap);
        }
        s_pre[NW] = sum;
    }
    __syncthreads();
    const int total = s_pre[NW];
    if (total == 0) return;
    for (int i = threadIdx.x; i < 2 * JT_ELEMS; i += blockDim.x) reinterpret_cast<unsigned*>(sJc)[i] = 0u;
    const int ntx = A.g.nt[0], nty = A.g.nt[1];
    const int tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
    tile_flush_index(A, tx * TILE, ty * TILE, tz * TILE, s_gidx);
    if (threadIdx.x < NW) cnt[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t sJa = smem_u32(sJc);
    for (int k = threadIdx.x; k < total; k += blockDim.x) {
        int w = 0;
        while (w + 1 < NW && s_pre[w + 1] <= k) ++w;
        esk_record(A.esk_buf + (((size_t)tile * NW + w) * A.esk_wcap + (k - s_pre[w])) * ESK_WORDS, sJa);
    }
    __syncthreads();
    tile_flush_j<T, 256>(A, sJc, s_gidx);
}

// Before a step whose tiles are split over several CTAs: per tile, the output cell
// ranges (exclusive scan of the input histogram) into goff, the output histogram set to
// the input one (the CTAs then move the counts of the particles that change cell), the
// input count kept in cnt_in, the new count (the ranges' total) and zero holes.
template <typename T>
__global__ void __launch_bounds__(256) k_split_prep(PushArgs<T> A) {
    __shared__ int s_off[TILE_CELLS], s_hn[TILE_CELLS], s_wsum[8], s_total;
    const int tile = blockIdx.x;
    const int* hin = A.hin + (size_t)tile * TILE_CELLS;
    hist_scan<true>(hin, s_off, s_hn, s_wsum, &s_total);
    __syncthreads();
    for (int i = threadIdx.x; i < TILE_CELLS; i += blockDim.x) {
        A.goff[(size_t)tile * TILE_CELLS + i] = s_off[i];
        A.hout[(size_t)tile * TILE_CELLS + i] = s_hn[i];
    }
    if (threadIdx.x == 0) {
        A.cnt_in[tile] = A.pa.count[tile];
        A.pa.count[tile] = s_total;
        A.pa.holes[tile] = 0;
    }
}

// Spill-list particles: same arithmetic with global-memory gather and deposit.
template <typename T, bool RECK, bool ESK>
__global__ void __launch_bounds__(256) k_list_push(PushArgs<T> A) {
    const int n = min(A.ctr->spill_count[A.parity], A.spill_cap);
    double kacc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        Rec<T> r = A.spill[i];
        const int gx = r.cell % A.g.n[0], gy = (r.cell / A.g.n[0]) % A.g.n[1], gz = r.cell / (A.g.n[0] * A.g.n[1]);
        auto fetch = [&](int comp, int x, int y, int z) -> T {
            const T* a = comp < 3 ? A.f.E[comp] : A.f.B[comp - 3];
            return a[A.g.pidx(x, y, z)];
        };
        using Acc = typename JTraits<T>::acc_t;
        auto add = [&](int comp, int x, int y, int z, Acc v) {
            const int xx = x_after(A.g, x);
            if (v != Acc(0) && xx >= 0)
                acc_atomic(A.f.J[comp] + A.g.cidx(xx, wrap_idx(y, A.g.n[1]), wrap_idx(z, A.g.n[2])), v);
        };
        T Ep[3], Bp[3], u[3] = {r.u[0], r.u[1], r.u[2]}, d2[3];
        gather_eb<T>(fetch, gx, gy, gz, r.d[0], r.d[1], r.d[2], Ep, Bp);
        T gm1_old = T(0);
        if (RECK) gm1_old = gamma_minus_one(u);
        const T ig = boris(A.eps, Ep, Bp, u);
        if (!(ig > T(0))) atomicOr(&A.ctr->err, ERRB_NAN);
        if (RECK) kacc += (double)r.w * A.mass * 0.5 * ((double)gm1_old + (double)gamma_minus_one(u));
        int s[3];
        for (int k = 0; k < 3; ++k) {
            s[k] = advance(r.d[k], A.dtd[k] * u[k] * ig, d2[k]);
            if (s[k] > 1 || s[k] < -1) {
                atomicOr(&A.ctr->err, ERRB_SUPERLUMINAL);
                s[k] = s[k] > 0 ? 1 : -1;
            }
        }
        const T cw[3] = {A.cq[0] * r.w, A.cq[1] * r.w, A.cq[2] * r.w};
        if (ESK) esirkepov_deposit<T>(add, gx, gy, gz, r.d, s, d2, cw);
        else zigzag_deposit<T>(add, gx, gy, gz, r.d, s, d2, cw);
        int nxg = x_after(A.g, gx + s[0]);
        if (nxg >= 0) nxg -= A.xshift;   // a window move: the first column leaves
        if (nxg < 0) {   // left an open x face (or the window): removed
            atomicAdd(&A.ctr->escaped, 1);
            continue;
        }
        Rec<T> o;
        o.cell = (wrap_idx(gz + s[2], A.g.n[2]) * A.g.n[1] + wrap_idx(gy + s[1], A.g.n[1])) * A.g.n[0] + nxg;
        o.id = r.id;
        for (int k = 0; k < 3; ++k) {
            o.d[k] = d2[k];
            o.u[k] = u[k];
        }
        o.w = r.w;
        const int slot = atomicAdd(&A.ctr->mover_count[A.parity], 1);
        if (slot < A.mover_cap) A.movers[slot] = o;
        else atomicOr(&A.ctr->err, ERRB_OVERFLOW);
    }
    if (RECK) {
        for (int o = 16; o > 0; o >>= 1) kacc += __shfl_xor_sync(0xffffffffu, kacc, o);
        if ((threadIdx.x & 31) == 0 && kacc != 0.0) atomicAdd(A.krec, kacc);
    }
}

// Movers into the end of the segment of their new tile in the block the step writes
// (and into that tile's cell histogram); a full segment sends them to the spill list of
// the next step.  Also resets the counters of the other parity.
template <typename T, bool IDS>
__global__ void __launch_bounds__(256) k_append(PushArgs<T> A) {
    const int n = min(A.ctr->mover_count[A.parity], A.mover_cap);
    const int nxt = A.parity ^ 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.ctr->mover_count[nxt] = 0;       // consumed by the previous step's append
        A.ctr->spill_count[A.parity] = 0;  // consumed by this step's list push
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Rec<T> r = A.movers[i];
        const int gx = r.cell % A.g.n[0], gy = (r.cell / A.g.n[0]) % A.g.n[1], gz = r.cell / (A.g.n[0] * A.g.n[1]);
        const int tx = gx >> 3, ty = gy >> 3, tz = gz >> 3;
        const int t = (tz * A.g.nt[1] + ty) * A.g.nt[0] + tx;
        const int slot = atomicAdd(A.pb.count + t, 1);
        if (slot < A.pb.cap[t]) {
            const long long q = (long long)A.pb.seg_start[t] + slot;
            const int lc = (gx & 7) | ((gy & 7) << 3) | ((gz & 7) << 6);
            A.pb.cell[q] = lc;
            A.pb.d[0][q] = r.d[0];
            A.pb.d[1][q] = r.d[1];
            A.pb.d[2][q] = r.d[2];
            A.pb.u[0][q] = r.u[0];
            A.pb.u[1][q] = r.u[1];
            A.pb.u[2][q] = r.u[2];
            A.pb.w[q] = r.w;
            if (IDS) A.pb.id[q] = r.id;
            atomicAdd(A.hout + (size_t)t * TILE_CELLS + lc, 1);
        } else {
            const int sp = atomicAdd(&A.ctr->spill_count[nxt], 1);
            if (sp < A.spill_cap) A.spill[sp] = r;
            else atomicOr(&A.ctr->err, ERRB_OVERFLOW);
        }
    }
}

// Backward Boris half step u^0 -> u^{-1/2} (section 2.4) for the particles of the
// tile segments, with E^0 and B^0 read from global memory.
template <typename T>
__global__ void __launch_bounds__(256) k_backpush(PushArgs<T> A, const T* B0x, const T* B0y, const T* B0z) {
    const int ntile = A.g.nt[0] * A.g.nt[1] * A.g.nt[2];
    for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int cnt = min(A.pa.count[t], A.pa.cap[t]);
        const int tx = t % A.g.nt[0], ty = (t / A.g.nt[0]) % A.g.nt[1], tz = t / (A.g.nt[0] * A.g.nt[1]);
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const long long p = (long long)A.pa.seg_start[t] + i;
            const int lc = A.pa.cell[p];
            if (lc < 0) continue;
            const int gx = tx * TILE + (lc & 7), gy = ty * TILE + ((lc >> 3) & 7), gz = tz * TILE + (lc >> 6);
            auto fetch = [&](int comp, int x, int y, int z) -> T {
                const T* a = comp < 3 ? A.f.E[comp] : (comp == 3 ? B0x : comp == 4 ? B0y : B0z);
                return a[A.g.pidx(x, y, z)];
            };
            T Ep[3], Bp[3], u[3] = {A.pa.u[0][p], A.pa.u[1][p], A.pa.u[2][p]};
            gather_eb<T>(fetch, gx, gy, gz, A.pa.d[0][p], A.pa.d[1][p], A.pa.d[2][p], Ep, Bp);
            boris(A.eps, Ep, Bp, u);
            A.pa.u[0][p] = u[0];
            A.pa.u[1][p] = u[1];
            A.pa.u[2][p] = u[2];
        }
    }
}

// ---------------------------------------------------------------------------
// Moving window: the plasma of the window's new last column (section 4 set-up), at rest,
// into the mover list, from where the append places it in its tiles.  Particle t of the
// column (t = 0 .. m - 1) is, x fastest: x offset a (of the na offsets whose density is
// not zero), y offset b, z offset c, y cell j, z cell k; its id is id_base + t.
struct InjectArgs {
    int nx, ny, py, pz, na;
    long long m;
    long long id_base;
    double offx[MAX_WINDOW_PPCX];   // in-cell x offset of each active x offset
    double wx[MAX_WINDOW_PPCX];     // weight of a particle at it
};

template <typename T>
__global__ void __launch_bounds__(256) k_inject(PushArgs<T> A, InjectArgs I) {
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // whole warps iterate together (the counter reservation is a warp vote)
    for (long long t0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); t0 < I.m; t0 += stride) {
        const long long t = t0 + lane;
        const bool valid = t < I.m;
        const unsigned mm = __ballot_sync(0xffffffffu, valid);
        int base = 0;
        if (lane == 0) base = atomicAdd(&A.ctr->mover_count[A.parity], __popc(mm));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (!valid) continue;
        long long r = t;
        const int a = (int)(r % I.na);
        r /= I.na;
        const int b = (int)(r % I.py);
        r /= I.py;
        const int c = (int)(r % I.pz);
        r /= I.pz;
        const int j = (int)(r % I.ny), k = (int)(r / I.ny);
        Rec<T> rc;
        rc.cell = (k * I.ny + j) * I.nx + (I.nx - 1);
        rc.id = (int)(I.id_base + t);
        rc.d[0] = (T)I.offx[a];
        rc.d[1] = (T)((2.0 * b + 1.0) / (2.0 * I.py));
        rc.d[2] = (T)((2.0 * c + 1.0) / (2.0 * I.pz));
        rc.u[0] = rc.u[1] = rc.u[2] = T(0);
        rc.w = (T)I.wx[a];
        const int slot = base + lane;   // the valid lanes are the low ones
        if (slot < A.mover_cap) A.movers[slot] = rc;
        else atomicOr(&A.ctr->err, ERRB_OVERFLOW);
    }
}

// ---------------------------------------------------------------------------
// Host launchers.


template <typename T>
static PushArgs<T> make_args(pic_ctx* c, SpeciesDev& s, int parity, double* krec, double dt_scale) {
    PushArgs<T> A{};
    A.g = c->g;
    A.pa = arrays<T>(s);
    A.pb = arrays_alt<T>(s);
    A.hin = s.hist[s.cur];
    A.hout = s.hist[s.cur ^ 1];
    for (int k = 0; k < 3; ++k) {
        A.f.E[k] = static_cast<T*>(c->E[k]);
        A.f.B[k] = static_cast<T*>(c->B[k]);
        A.f.J[k] = static_cast<typename JTraits<T>::acc_t*>(c->J[k]);
    }
    const double dt = c->desc.dt * dt_scale;
    const double* d = c->desc.d;
    A.eps = (T)(s.q * dt / (2.0 * s.m));
    for (int k = 0; k < 3; ++k) A.dtd[k] = (T)(dt / d[k]);
    A.cq[0] = (T)(s.q / (dt * d[1] * d[2]) * c->jinv);
    A.cq[1] = (T)(s.q / (dt * d[2] * d[0]) * c->jinv);
    A.cq[2] = (T)(s.q / (dt * d[0] * d[1]) * c->jinv);
    A.movers = static_cast<Rec<T>*>(s.movers);
    A.mover_cap = s.mover_cap;
    A.spill = static_cast<Rec<T>*>(s.spill);
    A.spill_cap = s.spill_cap;
    A.ctr = s.ctr;
    A.parity = parity;
    A.krec = krec;
    A.mass = s.m;
    A.wait_polls = c->wait_polls >= 0 ? c->wait_polls : MBAR_MAX_POLLS;
    return A;
}

static int sm_count(pic_ctx* c) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, c->desc.device);
    return v > 0 ? v : 152;
}

template <typename T, bool IDS, bool RECK, bool ESK, bool SPLIT = false>
static pic_status launch_tile(pic_ctx* c, PushArgs<T>& A) {
    auto kern = k_tile_push<T, IDS, RECK, ESK, SPLIT>;
    const size_t smem = tile_smem_bytes<T>();
    GBPIC_CHECK(c, raise_smem_limit(reinterpret_cast<const void*>(kern), smem, c->desc.device));
    const int ntile = c->g.nt[0] * c->g.nt[1] * c->g.nt[2];
    LaunchScope ls(c, KC_TILE_PUSH);
    if (SPLIT) {
        k_split_prep<T><<<ntile, 256, 0, c->stream>>>(A);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    kern<<<ntile * (SPLIT ? A.parts : 1), Prec<T>::THREADS, smem, c->stream>>>(c->tmap[0], c->tmap[1], c->tmap[2],
                                                                            c->tmap[3], c->tmap[4], c->tmap[5], A);
    GBPIC_CHECK(c, cudaGetLastError());
    return PIC_OK;
}

// The moving window's new column for species s (host part of k_inject): the active x
// offsets and their weights from the density profile at the particles' absolute x.
template <typename T>
static pic_status inject_t(pic_ctx* c, SpeciesDev& s, PushArgs<T>& A) {
    const pic_window_desc& W = c->window;
    const Geom& g = c->g;
    const double* d = c->desc.d;
    InjectArgs I{};
    I.nx = g.n[0];
    I.ny = g.n[1];
    I.py = W.ppc[1];
    I.pz = W.ppc[2];
    const long long origin = c->window_moves + 1;   // cell 0 of the window after this move
    const int ppc = W.ppc[0] * W.ppc[1] * W.ppc[2];
    int na = 0;
    for (int a = 0; a < W.ppc[0]; ++a) {
        const double off = (2.0 * a + 1.0) / (2.0 * W.ppc[0]);
        const double X = (double)(origin + g.n[0] - 1) + off;
        double prof;
        if (W.ramp > 0) {
            const double r = (X - W.x0) / W.ramp;
            prof = W.density * (r < 0.0 ? 0.0 : (r > 1.0 ? 1.0 : r));
        } else {
            prof = X >= W.x0 ? W.density : 0.0;
        }
        const double w = prof * d[0] * d[1] * d[2] / ppc;
        if (w > 0) {
            I.offx[na] = off;
            I.wx[na] = w;
            ++na;
        }
    }
    I.na = na;
    I.m = (long long)na * W.ppc[1] * W.ppc[2] * g.n[1] * g.n[2];
    if (I.m == 0) return PIC_OK;
    I.id_base = s.n_loaded + s.n_injected;
    if (c->desc.track_ids && I.id_base + I.m > 0x7fffffffLL) {
        c->err = "moving window: more than 2^31 particle ids";
        return PIC_ERR_TILE_OVERFLOW;
    }
    {
        LaunchScope ls(c, KC_OTHER);
        const long long blocks = std::min<long long>((I.m + 255) / 256, 8LL * sm_count(c));
        k_inject<T><<<(unsigned)blocks, 256, 0, c->stream>>>(A, I);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    s.n_injected += I.m;
    return PIC_OK;
}

// Esirkepov's crossers' export segments of species s, per tile and warp: every
// particle the warp can step (its rows of 32 R slots of the largest tile capacity), so
// that none can fill.  Reserved once, before the species' first Esirkepov step.
template <typename T>
static pic_status reserve_esk_t(pic_ctx* c, SpeciesDev& s) {
    if (s.esk_buf) return PIC_OK;
    constexpr int NWT = Prec<T>::THREADS / 32, ROW = 32 * Prec<T>::R;
    int maxcap = 0;
    for (int cap : s.h_cap) maxcap = std::max(maxcap, cap);
    const int rows = (maxcap + ROW - 1) / ROW;
    const int wcap = std::max(1, (rows + NWT - 1) / NWT) * ROW;
    const size_t nseg = (size_t)c->g.nt[0] * c->g.nt[1] * c->g.nt[2] * NWT;
    const size_t bytes = nseg * (size_t)wcap * ESK_WORDS * sizeof(T);
    void* buf = dev_alloc(c, bytes);
    int* cnt = buf ? static_cast<int*>(dev_alloc(c, nseg * sizeof(int))) : nullptr;
    if (!cnt) {
        if (buf) dev_free(c, buf);
        c->err = "Esirkepov's deposit: no device memory for the crossers' records (" + std::to_string(bytes) + " bytes)";
        return PIC_ERR_OOM;
    }
    GBPIC_CHECK(c, cudaMemsetAsync(cnt, 0, nseg * sizeof(int), c->stream));
    s.esk_buf = buf;
    s.esk_cnt = cnt;
    s.esk_wcap = wcap;
    return PIC_OK;
}

pic_status reserve_esk_records(pic_ctx* c, SpeciesDev& s) {
    return c->prec == PIC_FP64 ? reserve_esk_t<double>(c, s) : reserve_esk_t<float>(c, s);
}

template <typename T>
static pic_status push_species_t(pic_ctx* c, SpeciesDev& s, int parity, double* krec, int xshift, bool inject) {
    PushArgs<T> A = make_args<T>(c, s, parity, krec, 1.0);
    A.xshift = xshift;
    const bool ids = c->desc.track_ids != 0, rec = krec != nullptr;
    pic_status st;
    const bool esk = c->deposit == PIC_DEPOSIT_ESIRKEPOV;
    const bool tsc = c->shape == PIC_SHAPE_TSC;
    {   // a grid of fewer tiles than SMs splits each tile's rows over several CTAs (the
        // ZigZag kernel), up to two CTAs per SM and at least one row of slots per CTA
        const int ntile = c->g.nt[0] * c->g.nt[1] * c->g.nt[2];
        const int sms = sm_count(c);
        A.parts = 1;
        if (!esk && !tsc && ntile < sms) {
            int maxcap = 0;
            for (int cap : s.h_cap) maxcap = std::max(maxcap, cap);
            const int rows = (maxcap + 32 * Prec<T>::R - 1) / (32 * Prec<T>::R);
            A.parts = std::max(1, std::min((2 * sms + ntile - 1) / ntile, rows));
        }
        if (A.parts > 1) {
            if (!s.split_buf) {
                s.split_buf = static_cast<int*>(dev_alloc(c, sizeof(int) * (size_t)ntile * (TILE_CELLS + 1)));
                if (!s.split_buf) return PIC_ERR_OOM;
            }
            A.goff = s.split_buf;
            A.cnt_in = s.split_buf + (size_t)ntile * TILE_CELLS;
        }
    }
    const int ntile_all = c->g.nt[0] * c->g.nt[1] * c->g.nt[2];
    if (esk && !tsc && !s.esk_buf) {
        c->err = "Esirkepov's deposit: the crossers' record list is not reserved";
        return PIC_ERR_STATE;
    }
    if (esk) {
        A.esk_buf = static_cast<T*>(s.esk_buf);
        A.esk_cnt = s.esk_cnt;
        A.esk_wcap = s.esk_wcap;
    }
    if (tsc) {
        st = launch_tsc_push<T>(c, A, ids, rec);   // its tile step and spill-list step
    } else if (esk) {
        if (ids) st = rec ? launch_tile<T, true, true, true>(c, A) : launch_tile<T, true, false, true>(c, A);
        else st = rec ? launch_tile<T, false, true, true>(c, A) : launch_tile<T, false, false, true>(c, A);
        if (st == PIC_OK) {
            LaunchScope ls(c, KC_ESK);
            k_esk_crossers<T><<<ntile_all, 256, 8 * JT_ELEMS, c->stream>>>(A);
            GBPIC_CHECK(c, cudaGetLastError());
        }
    } else if (A.parts > 1) {   // fewer tiles than SMs: several CTAs per tile
        if (ids) st = rec ? launch_tile<T, true, true, false, true>(c, A) : launch_tile<T, true, false, false, true>(c, A);
        else st = rec ? launch_tile<T, false, true, false, true>(c, A) : launch_tile<T, false, false, false, true>(c, A);
    } else {
        if (ids) st = rec ? launch_tile<T, true, true, false>(c, A) : launch_tile<T, true, false, false>(c, A);
        else st = rec ? launch_tile<T, false, true, false>(c, A) : launch_tile<T, false, false, false>(c, A);
    }
    if (st != PIC_OK) return st;
    const int grid = 2 * sm_count(c);
    if (!tsc) {
        LaunchScope ls(c, KC_LIST_PUSH);
        if (esk) {
            if (rec) k_list_push<T, true, true><<<grid, 256, 0, c->stream>>>(A);
            else k_list_push<T, false, true><<<grid, 256, 0, c->stream>>>(A);
        } else {
            if (rec) k_list_push<T, true, false><<<grid, 256, 0, c->stream>>>(A);
            else k_list_push<T, false, false><<<grid, 256, 0, c->stream>>>(A);
        }
        GBPIC_CHECK(c, cudaGetLastError());
    }
    if (inject) {
        st = inject_t<T>(c, s, A);
        if (st != PIC_OK) return st;
    }
    {
        LaunchScope ls(c, KC_APPEND);
        if (ids) k_append<T, true><<<grid, 256, 0, c->stream>>>(A);
        else k_append<T, false><<<grid, 256, 0, c->stream>>>(A);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    s.cur ^= 1;   // the block just written holds the particles now
    return PIC_OK;
}

pic_status launch_push_species(pic_ctx* c, SpeciesDev& s, int parity, double* krec, int xshift, bool inject) {
    return c->prec == PIC_FP64 ? push_species_t<double>(c, s, parity, krec, xshift, inject)
                               : push_species_t<float>(c, s, parity, krec, xshift, inject);
}

template <typename T>
static pic_status backpush_t(pic_ctx* c, SpeciesDev& s) {
    // B^0 = B^{-1/2} - dt/2 curl E^0 into scratch arrays, then a Boris step of -dt/2
    const size_t bytes = (size_t)c->g.padded_size() * sizeof(T);
    T* B0[3];
    for (int k = 0; k < 3; ++k) {
        B0[k] = static_cast<T*>(dev_alloc(c, bytes));
        if (!B0[k]) return PIC_ERR_OOM;
        GBPIC_CHECK(c, cudaMemcpyAsync(B0[k], c->B[k], bytes, cudaMemcpyDeviceToDevice, c->stream));
    }
    void* saved[3] = {c->B[0], c->B[1], c->B[2]};
    for (int k = 0; k < 3; ++k) c->B[k] = B0[k];
    pic_status st = launch_faraday_half(c, nullptr);
    for (int k = 0; k < 3; ++k) c->B[k] = saved[k];
    if (st != PIC_OK) return st;
    PushArgs<T> A = make_args<T>(c, s, 0, nullptr, -0.5);
    if (c->shape == PIC_SHAPE_TSC) {
        st = launch_tsc_backpush<T>(c, A, static_cast<const T*>(B0[0]), static_cast<const T*>(B0[1]),
                                    static_cast<const T*>(B0[2]));
        if (st != PIC_OK) return st;
    } else {
        LaunchScope ls(c, KC_OTHER);
        k_backpush<T><<<4 * sm_count(c), 256, 0, c->stream>>>(A, B0[0], B0[1], B0[2]);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    GBPIC_CHECK(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 3; ++k) dev_free(c, B0[k]);
    return PIC_OK;
}

pic_status launch_backpush(pic_ctx* c, SpeciesDev& s) {
    return c->prec == PIC_FP64 ? backpush_t<double>(c, s) : backpush_t<float>(c, s);
}

}  // namespace gbpic

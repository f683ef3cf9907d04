// Particle step with the quadratic particle shape (section 2.5, Eq. (16) with the
// first-order B-spline cloud b1, a triangle two cells wide; section 5 lists
// higher-order shapes as an extension of the paper's CIC scheme).  The cloud's overlap
// with the unit cell around a sample point gives the quadratic B-spline weight of the
// triangular-shaped cloud (TSC) for a sample at distance r (cell units):
//   W2(r) = 3/4 - r^2 (|r| <= 1/2),  (3/2 - |r|)^2 / 2 (1/2 <= |r| <= 3/2),  0 beyond.
// Every field component is interpolated from its own Yee location with the three
// nearest samples per dimension (27 per component), and the current is Esirkepov's
// (Esirkepov 2001) with the same shape on the four nodes per dimension that the move
// touches, so the discrete continuity equation holds exactly against the TSC charge.
//
//   k_tsc_tile_push   one CTA per 8^3-cell tile on the same tile segments, output
//                     regrouping, mover list and spill list as the CIC step: E, B of
//                     local cells -1..9 staged in shared memory (periodic wrap), the
//                     current in a shared fixed-point J tile of local edges/nodes
//                     -2..10, flushed to HBM with integer (FP32) or FP64 atomics.
//   k_tsc_list_push   the spill list's particles with global-memory gather and deposit.
// The shape supports periodic boundaries (the host rejects an open x).
#include <type_traits>

#include "push_common.cuh"

namespace gbpic {

constexpr int TSF = 11;                   // staged field extent per dimension: local -1..9
constexpr int TSF3 = TSF * TSF * TSF;
constexpr int TSJ = 13;                   // J tile extent per dimension: local -2..10
constexpr int TSJ3 = TSJ * TSJ * TSJ;
constexpr int TSJ_ELEMS = 3 * TSJ3;
constexpr int TSC_THREADS = 256;
constexpr int TSC_WARPS = TSC_THREADS / 32;

template <typename T> __host__ __device__ constexpr size_t tsc_smem_bytes() {
    // staged fields, J tile (8 bytes per element), the warps' staged movers, + 128 for
    // the alignment of the dynamic base
    return align128((size_t)6 * TSF3 * sizeof(T)) + align128((size_t)TSJ_ELEMS * 8) +
           align128((size_t)TSC_WARPS * MQ * sizeof(Rec<T>)) + 128;
}

template <typename T> __device__ __forceinline__ T tsc_w(T r) {
    r = r < T(0) ? -r : r;
    if (r <= T(0.5)) return T(0.75) - r * r;
    const T a = T(1.5) - r;
    return r < T(1.5) ? T(0.5) * a * a : T(0);
}

// W2(r + D) - W2(r) without subtracting two weights (which would leave an absolute
// rounding error of the weights' size, large against the change of a short move): on
// each quadratic piece of W2 the difference is written with D as a factor, and a move
// that crosses a piece boundary (at most one: the pieces are one cell wide and |D| < 1)
// is split there.  Pieces: q = -2 (r < -3/2), -1 (W = (3/2 + r)^2 / 2), 0 (W = 3/4 - r^2),
// 1 (W = (3/2 - r)^2 / 2), 2 (r >= 3/2).
template <typename T> __device__ __forceinline__ int tsc_piece(T r) {
    const int q = (int)floor(r + T(0.5));
    return q < -2 ? -2 : (q > 2 ? 2 : q);
}
template <typename T> __device__ __forceinline__ T tsc_dpiece(int q, T a, T D) {
    if (q == 0) return -D * (T(2) * a + D);
    if (q == 1) return T(-0.5) * D * (T(3) - T(2) * a - D);
    if (q == -1) return T(0.5) * D * (T(3) + T(2) * a + D);
    return T(0);
}
template <typename T> __device__ __forceinline__ T tsc_dw(T r, T D) {
    const int qa = tsc_piece(r), qb = tsc_piece(r + D);
    if (qa == qb) return tsc_dpiece(qa, r, D);
    const T rb = T(qa < qb ? qa : qb) + T(0.5);   // the boundary between the two pieces
    const T D1 = rb - r;
    return tsc_dpiece(qa, r, D1) + tsc_dpiece(qb, rb, D - D1);
}

// Weights of the three samples nearest a particle at in-cell offset d (0 <= d < 1):
// a node-located component samples local indices base .. base + 2 with base = m - 1, m
// the nearest node (0 or 1); a half-located one samples -1 .. 1 (the sample of index i
// sits at i + 1/2).
template <typename T> __device__ __forceinline__ void tsc_node(T d, int& base, T w[3]) {
    const int m = d >= T(0.5) ? 1 : 0;
    const T e = d - T(m);   // offset from the nearest node, -1/2 <= e < 1/2
    base = m - 1;
    const T a = T(0.5) - e, b = T(0.5) + e;
    w[0] = T(0.5) * a * a;
    w[1] = T(0.75) - e * e;
    w[2] = T(0.5) * b * b;
}
template <typename T> __device__ __forceinline__ void tsc_half(T d, T w[3]) {
    const T e = d - T(0.5);
    const T a = T(0.5) - e, b = T(0.5) + e;
    w[0] = T(0.5) * a * a;
    w[1] = T(0.75) - e * e;
    w[2] = T(0.5) * b * b;
}

// 27-point interpolation of one component from F(i, j, k) (any fetch), the first
// samples at (x0, y0, z0).
template <typename T, typename Fetch>
__device__ __forceinline__ T interp27(Fetch F, int x0, int y0, int z0, const T wx[3], const T wy[3], const T wz[3]) {
    T v = T(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T vc = T(0);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const T vb = wx[0] * F(x0, y0 + b, z0 + c) + wx[1] * F(x0 + 1, y0 + b, z0 + c) + wx[2] * F(x0 + 2, y0 + b, z0 + c);
            vc += wy[b] * vb;
        }
        v += wz[c] * vc;
    }
    return v;
}

// E and B at a particle in cell (x, y, z) with offsets (dx, dy, dz); Fc(comp) returns a
// fetch of component comp (E 0..2, B 3..5) over the indices (i, j, k).
template <typename T, typename FetchC>
__device__ __forceinline__ void gather_tsc(FetchC Fc, int x, int y, int z, T dx, T dy, T dz, T Ep[3], T Bp[3]) {
    int bx, by, bz;
    T nx[3], ny[3], nz[3], hx[3], hy[3], hz[3];
    tsc_node(dx, bx, nx);
    tsc_node(dy, by, ny);
    tsc_node(dz, bz, nz);
    tsc_half(dx, hx);
    tsc_half(dy, hy);
    tsc_half(dz, hz);
    // E_c is half-located along c; B_c along the two other dimensions
    Ep[0] = interp27<T>(Fc(0), x - 1, y + by, z + bz, hx, ny, nz);
    Ep[1] = interp27<T>(Fc(1), x + bx, y - 1, z + bz, nx, hy, nz);
    Ep[2] = interp27<T>(Fc(2), x + bx, y + by, z - 1, nx, ny, hz);
    Bp[0] = interp27<T>(Fc(3), x + bx, y - 1, z - 1, nx, hy, hz);
    Bp[1] = interp27<T>(Fc(4), x - 1, y + by, z - 1, hx, ny, hz);
    Bp[2] = interp27<T>(Fc(5), x - 1, y - 1, z + bz, hx, hy, nz);
}

// Esirkepov's deposit with the TSC shape for a move from offsets d1 in the start cell
// to offsets d2 in the cell s away (|s_d| <= 1).  Per dimension, relative to the start
// cell, X1 = d1 and X2 = s + d2; the support is the nodes b .. b + 3 with b = min(m1,
// m2) - 1 (m the node nearest to X), S0 and S1 the node weights before and after, DS =
// S1 - S0 (tsc_dw);  Wx = DSx (S0y S0z + DSy S0z / 2 + S0y DSz / 2 + DSy DSz / 3) (y, z
// cyclically), and Jx at the edge b + i + 1/2 (i = 0..2) is -cw_x times the sum of Wx
// over the nodes b .. b + i.  Add(comp, ox, oy, oz, v) receives each non-zero value v
// (working precision, fixed-point units on the FP32 path) with the offsets of the
// component's location from the start cell.
// Along a dimension whose nearest node did not change (m1 = m2) the fourth node b + 3
// carries neither weight (it lies 3/2 or more from both positions, where W2 and its
// change vanish exactly), and the third edge carries the sum of the three weight
// changes, zero but for rounding: both are skipped unless the nearest node changed.
template <typename T, typename AddFn>
__device__ __forceinline__ void esirkepov_tsc(AddFn Add, const T d1[3], const int s[3], const T d2[3], const T cw[3]) {
    int b[3];
    bool wide[3];
    T S0[3][4], DS[3][4];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T X1 = d1[k], X2 = T(s[k]) + d2[k];
        // the move X2 - X1 from the stored offsets, in the order that keeps it exact for
        // a short move (1 - d1 and d2 - 1 are exact near a face)
        const T D = s[k] == 0 ? d2[k] - d1[k] : (s[k] > 0 ? (T(1) - d1[k]) + d2[k] : (d2[k] - T(1)) - d1[k]);
        const int m1 = X1 >= T(0.5) ? 1 : 0;
        const int m2 = (int)floor(X2 + T(0.5));
        b[k] = min(m1, m2) - 1;
        wide[k] = m1 != m2;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const T r = X1 - T(b[k] + j);
            S0[k][j] = tsc_w(r);
            DS[k][j] = tsc_dw(r, D);
        }
    }
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
        const int p = comp == 2 ? 0 : comp + 1, r = comp == 0 ? 2 : comp - 1;
#pragma unroll
        for (int jp = 0; jp < 4; ++jp) {
            if (jp == 3 && !wide[p]) continue;
#pragma unroll
            for (int jr = 0; jr < 4; ++jr) {
                if (jr == 3 && !wide[r]) continue;
                const T t = S0[p][jp] * S0[r][jr] + T(0.5) * DS[p][jp] * S0[r][jr] + T(0.5) * S0[p][jp] * DS[r][jr] +
                            DS[p][jp] * DS[r][jr] * T(1.0 / 3.0);
                if (t == T(0)) continue;
                T acc = T(0);
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    if (i == 2 && !wide[comp]) continue;
                    acc += DS[comp][i] * t;
                    const T v = -cw[comp] * acc;
                    if (v == T(0)) continue;
                    int o[3];
                    o[comp] = b[comp] + i;
                    o[p] = b[p] + jp;
                    o[r] = b[r] + jr;
                    Add(comp, o[0], o[1], o[2], v);
                }
            }
        }
    }
}

// Shared J tile element (comp, local x, y, z), local -2..10.
__device__ __forceinline__ int tsc_j_index(int comp, int x, int y, int z) {
    return comp * TSJ3 + ((z + 2) * TSJ + (y + 2)) * TSJ + (x + 2);
}

// Add v (fixed-point units) to a split 32-bit element of the J tile (the layout of
// tile_add: lo word at e, hi word at NE + e, element = hi * 2^20 + lo, lo in [0, 2^20]
// per term).  A deposit element here can receive more terms in one tile step than the
// 4096 that keep a lo word below 2^32, so the tile kernel folds the lo words into the
// hi words (tsc_fold) after every TSC_FOLD particles: at most TSC_FOLD terms reach a
// word between two folds, and the adds stay reductions that return nothing.
constexpr int TSC_FOLD_ITERS = 15;                        // loop iterations between folds
constexpr int TSC_FOLD = TSC_FOLD_ITERS * TSC_THREADS;    // 3840 particles: lo < 2^20 (3841)
static_assert(TSC_FOLD < 4095, "a lo word holds the terms between two folds");
__device__ __forceinline__ void tsc_tile_add(unsigned* words, int e, float v) {
    const float hf = floorf(v * 9.5367431640625e-07f);   // v / 2^20
    const int hi = __float2int_rz(hf);
    const unsigned lo = (unsigned)__float2int_rn(__fmaf_rn(hf, -1048576.0f, v));
    // (the atomics are left to the compiler, without a memory clobber, so that the
    // independent adds of one particle overlap instead of waiting one by one)
    atomicAdd(words + e, lo);
    atomicAdd(words + TSJ_ELEMS + e, (unsigned)hi);
}
__device__ __forceinline__ void tsc_tile_add(double* vals, int e, double v) { atomicAdd(vals + e, v); }
// hi += lo >> 20, lo &= 2^20 - 1 for every element (block-wide, between barriers): the
// element hi * 2^20 + lo keeps its value.
__device__ __forceinline__ void tsc_fold(unsigned* words) {
    for (int e = threadIdx.x; e < TSJ_ELEMS; e += TSC_THREADS) {
        const unsigned lo = words[e];
        if (lo >> 20) {
            words[e] = lo & 0xFFFFFu;
            words[TSJ_ELEMS + e] += lo >> 20;
        }
    }
}
__device__ __forceinline__ void tsc_fold(double*) {}

template <typename T, bool IDS, bool RECK>
__global__ void __launch_bounds__(TSC_THREADS, sizeof(T) == sizeof(float) ? 2 : 1) k_tsc_tile_push(PushArgs<T> A) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    using Acc = typename JTraits<T>::acc_t;
    constexpr int NT = TSC_THREADS;
    T* sF = reinterpret_cast<T*>(smem);
    unsigned char* sJ = smem + align128((size_t)6 * TSF3 * sizeof(T));
    // the J tile's words: two 32-bit halves per element (FP32) or one double (FP64)
    using JW = typename std::conditional<JTraits<T>::fixed, unsigned, double>::type;
    JW* sJw = reinterpret_cast<JW*>(sJ);
    Rec<T>* sM = reinterpret_cast<Rec<T>*>(sJ + align128((size_t)TSJ_ELEMS * 8)) + (threadIdx.x >> 5) * MQ;
    __shared__ int s_off[TILE_CELLS];
    __shared__ int s_hn[TILE_CELLS];
    __shared__ int s_wsum[8];
    __shared__ int s_total, s_left;
    __shared__ int s_gidx[3 * TSJ];

    const int tile = blockIdx.x;
    const int cnt = min(A.pa.count[tile], A.pa.cap[tile]);
    const int* hin = A.hin + (size_t)tile * TILE_CELLS;
    int* hout = A.hout + (size_t)tile * TILE_CELLS;
    const int lane = threadIdx.x & 31;
    if (cnt == 0) {
        for (int i = threadIdx.x; i < TILE_CELLS; i += NT) hout[i] = 0;
        if (threadIdx.x == 0) A.pa.holes[tile] = 0;
        return;
    }
    const int ntx = A.g.nt[0], nty = A.g.nt[1];
    const int tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
    const int ox = tx * TILE, oy = ty * TILE, oz = tz * TILE;
    const int n0 = A.g.n[0], n1 = A.g.n[1], n2 = A.g.n[2];

    if (threadIdx.x == 0) s_left = 0;
    // E, B of local cells -1..9 (periodic wrap), the J tile cleared, the output ranges
    for (int e = threadIdx.x; e < 6 * TSF3; e += NT) {
        const int c = e / TSF3, r = e - c * TSF3;
        const int lz = r / (TSF * TSF), r2 = r - lz * (TSF * TSF);
        const int ly = r2 / TSF, lx = r2 - ly * TSF;
        const T* F = c < 3 ? A.f.E[c] : A.f.B[c - 3];
        sF[e] = F[A.g.pidx(wrap_idx(ox + lx - 1, n0), wrap_idx(oy + ly - 1, n1), wrap_idx(oz + lz - 1, n2))];
    }
    {
        unsigned long long* z = reinterpret_cast<unsigned long long*>(sJ);
        for (int i = threadIdx.x; i < TSJ_ELEMS; i += NT) z[i] = 0ull;
    }
    if (threadIdx.x < 3 * TSJ) {
        const int d = threadIdx.x / TSJ, l = threadIdx.x - d * TSJ - 2;
        s_gidx[threadIdx.x] = d == 0 ? x_after(A.g, ox + l) : (d == 1 ? wrap_idx(oy + l, n1) : wrap_idx(oz + l, n2));
    }
    hist_scan(hin, s_off, s_hn, s_wsum, &s_total);
    __syncthreads();

    const int ext[3] = {min(TILE, n0 - ox), min(TILE, n1 - oy), min(TILE, n2 - oz)};
    const int seg = A.pa.seg_start[tile];
    double kacc = 0.0;
    int left = 0, esc = 0, mq = 0;
    auto fetch = [&](int comp) {
        const T* F = sF + comp * TSF3;
        return [F](int i, int j, int k) -> T { return F[((k + 1) * TSF + (j + 1)) * TSF + (i + 1)]; };
    };
    // whole warps step together (the mover staging is a warp vote), and the whole block
    // runs the same iterations (the FP32 tile's folds are block-wide)
    int iter = 0;
    for (int base = 0; base < cnt; base += NT) {
        if constexpr (JTraits<T>::fixed) {
            if (++iter > TSC_FOLD_ITERS) {
                iter = 1;
                __syncthreads();
                tsc_fold(sJw);
                __syncthreads();
            }
        }
        const int i = base + threadIdx.x;
        const int p = seg + i;
        const int lc = i < cnt ? __ldcg(A.pa.cell + p) : HOLE;
        const bool active = lc >= 0;
        int s[3] = {0, 0, 0};
        int x = 0, y = 0, z = 0;
        T u[3] = {T(0), T(0), T(0)}, d2[3] = {T(0), T(0), T(0)}, w = T(0);
        bool move = false;
        int nlc = -1;
        if (active) {
            x = lc & 7;
            y = (lc >> 3) & 7;
            z = lc >> 6;
            const T d1[3] = {__ldcg(A.pa.d[0] + p), __ldcg(A.pa.d[1] + p), __ldcg(A.pa.d[2] + p)};
            u[0] = __ldcg(A.pa.u[0] + p);
            u[1] = __ldcg(A.pa.u[1] + p);
            u[2] = __ldcg(A.pa.u[2] + p);
            w = __ldcg(A.pa.w + p);
            T Ep[3], Bp[3];
            gather_tsc<T>(fetch, x, y, z, d1[0], d1[1], d1[2], Ep, Bp);
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
            const T cw[3] = {A.cq[0] * w, A.cq[1] * w, A.cq[2] * w};
            esirkepov_tsc<T>(
                [&](int comp, int ax, int ay, int az, T v) { tsc_tile_add(sJw, tsc_j_index(comp, x + ax, y + ay, z + az), v); },
                d1, s, d2, cw);
            const int nx = x + s[0], ny = y + s[1], nz = z + s[2];
            const bool stay = nx >= 0 && nx < ext[0] && ny >= 0 && ny < ext[1] && nz >= 0 && nz < ext[2];
            move = !stay;
            if (stay) nlc = nx | (ny << 3) | (nz << 6);
            const int o = seg + atomicAdd(&s_off[lc], 1);
            __stcs(A.pb.cell + o, stay ? nlc : HOLE);
            if (stay) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    __stcs(A.pb.d[k] + o, d2[k]);
                    __stcs(A.pb.u[k] + o, u[k]);
                }
                __stcs(A.pb.w + o, w);
                if (IDS) __stcs(A.pb.id + o, __ldg(A.pa.id + p));
                atomicAdd(&s_hn[nlc], 1);
            } else {
                ++left;
            }
        }
        int gxm = 0;
        if (move) {
            gxm = x_after(A.g, ox + x + s[0]);
            if (gxm < 0) {   // left an open x face: removed
                move = false;
                ++esc;
            }
        }
        if (const unsigned mm = __ballot_sync(0xffffffffu, move)) {
            if (mq + __popc(mm) > MQ) movers_flush(A, sM, mq, lane);
            if (move) {
                Rec<T>& rc = sM[mq + __popc(mm & ((1u << lane) - 1u))];
                rc.cell = (wrap_idx(oz + z + s[2], n2) * n1 + wrap_idx(oy + y + s[1], n1)) * n0 + gxm;
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
    if (mq) movers_flush(A, sM, mq, lane);
    left = __reduce_add_sync(0xffffffffu, left);
    esc = __reduce_add_sync(0xffffffffu, esc);
    if (lane == 0 && left) atomicAdd(&s_left, left);
    if (lane == 0 && esc) atomicAdd(&A.ctr->escaped, esc);
    __syncthreads();
    for (int i = threadIdx.x; i < TILE_CELLS; i += NT) hout[i] = s_hn[i];
    if (threadIdx.x == 0) {
        A.pa.count[tile] = s_total;
        A.pa.holes[tile] = s_left;
    }
    // the J tile into HBM (the guard layers wrap onto the other side of the box)
    for (int e = threadIdx.x; e < TSJ_ELEMS; e += NT) {
        Acc v;
        if constexpr (JTraits<T>::fixed) {
            const unsigned* wd = reinterpret_cast<const unsigned*>(sJ);
            v = ((long long)(int)wd[TSJ_ELEMS + e] << 20) + (long long)wd[e];
        } else {
            v = reinterpret_cast<const double*>(sJ)[e];
        }
        if (v == Acc(0)) continue;
        const int comp = e / TSJ3, r = e - comp * TSJ3;
        const int lz = r / (TSJ * TSJ), r2 = r - lz * (TSJ * TSJ);
        const int ly = r2 / TSJ, lx = r2 - ly * TSJ;
        const int gx = s_gidx[lx];
        if (gx < 0) continue;
        acc_atomic(A.f.J[comp] + A.g.cidx(gx, s_gidx[TSJ + ly], s_gidx[2 * TSJ + lz]), v);
    }
    if (RECK) block_add_double(kacc, A.krec);
}

// Spill-list particles: the same step with global-memory gather and deposit.
template <typename T, bool RECK>
__global__ void __launch_bounds__(256) k_tsc_list_push(PushArgs<T> A) {
    const int n = min(A.ctr->spill_count[A.parity], A.spill_cap);
    const int n0 = A.g.n[0], n1 = A.g.n[1], n2 = A.g.n[2];
    double kacc = 0.0;
    using Acc = typename JTraits<T>::acc_t;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Rec<T> r = A.spill[i];
        const int gx = r.cell % n0, gy = (r.cell / n0) % n1, gz = r.cell / (n0 * n1);
        auto fetch = [&](int comp) {
            const T* F = comp < 3 ? A.f.E[comp] : A.f.B[comp - 3];
            const Geom& g = A.g;
            return [F, &g, n0, n1, n2](int x, int y, int z) -> T {
                return F[g.pidx(wrap_idx(x, n0), wrap_idx(y, n1), wrap_idx(z, n2))];
            };
        };
        T Ep[3], Bp[3], u[3] = {r.u[0], r.u[1], r.u[2]}, d2[3];
        gather_tsc<T>(fetch, gx, gy, gz, r.d[0], r.d[1], r.d[2], Ep, Bp);
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
        esirkepov_tsc<T>(
            [&](int comp, int ax, int ay, int az, T v) {
                const int xx = x_after(A.g, gx + ax);
                if (xx >= 0) acc_atomic(A.f.J[comp] + A.g.cidx(xx, wrap_idx(gy + ay, n1), wrap_idx(gz + az, n2)), (Acc)to_acc(v));
            },
            r.d, s, d2, cw);
        const int nxg = x_after(A.g, gx + s[0]);
        if (nxg < 0) {
            atomicAdd(&A.ctr->escaped, 1);
            continue;
        }
        Rec<T> o;
        o.cell = (wrap_idx(gz + s[2], n2) * n1 + wrap_idx(gy + s[1], n1)) * n0 + nxg;
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

// Backward Boris half step u^0 -> u^{-1/2} with the TSC gather (E^0 and B^0 from
// global memory).
template <typename T>
__global__ void __launch_bounds__(256) k_tsc_backpush(PushArgs<T> A, const T* B0x, const T* B0y, const T* B0z) {
    const int ntile = A.g.nt[0] * A.g.nt[1] * A.g.nt[2];
    const int n0 = A.g.n[0], n1 = A.g.n[1], n2 = A.g.n[2];
    for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int cnt = min(A.pa.count[t], A.pa.cap[t]);
        const int tx = t % A.g.nt[0], ty = (t / A.g.nt[0]) % A.g.nt[1], tz = t / (A.g.nt[0] * A.g.nt[1]);
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const long long p = (long long)A.pa.seg_start[t] + i;
            const int lc = A.pa.cell[p];
            if (lc < 0) continue;
            const int gx = tx * TILE + (lc & 7), gy = ty * TILE + ((lc >> 3) & 7), gz = tz * TILE + (lc >> 6);
            auto fetch = [&](int comp) {
                const T* F = comp < 3 ? A.f.E[comp] : (comp == 3 ? B0x : comp == 4 ? B0y : B0z);
                const Geom& g = A.g;
                return [F, &g, n0, n1, n2](int x, int y, int z) -> T {
                    return F[g.pidx(wrap_idx(x, n0), wrap_idx(y, n1), wrap_idx(z, n2))];
                };
            };
            T Ep[3], Bp[3], u[3] = {A.pa.u[0][p], A.pa.u[1][p], A.pa.u[2][p]};
            gather_tsc<T>(fetch, gx, gy, gz, A.pa.d[0][p], A.pa.d[1][p], A.pa.d[2][p], Ep, Bp);
            boris(A.eps, Ep, Bp, u);
            A.pa.u[0][p] = u[0];
            A.pa.u[1][p] = u[1];
            A.pa.u[2][p] = u[2];
        }
    }
}

// ---------------------------------------------------------------------------
// Host launchers.

template <typename T, bool IDS, bool RECK>
static pic_status launch_tsc_tile(pic_ctx* c, PushArgs<T>& A) {
    auto kern = k_tsc_tile_push<T, IDS, RECK>;
    const size_t smem = tsc_smem_bytes<T>();
    GBPIC_CHECK(c, raise_smem_limit(reinterpret_cast<const void*>(kern), smem, c->desc.device));
    const int ntile = c->g.nt[0] * c->g.nt[1] * c->g.nt[2];
    LaunchScope ls(c, KC_TILE_PUSH);
    kern<<<ntile, TSC_THREADS, smem, c->stream>>>(A);
    GBPIC_CHECK(c, cudaGetLastError());
    return PIC_OK;
}

template <typename T> pic_status launch_tsc_push(pic_ctx* c, PushArgs<T>& A, bool ids, bool rec) {
    pic_status st = ids ? (rec ? launch_tsc_tile<T, true, true>(c, A) : launch_tsc_tile<T, true, false>(c, A))
                        : (rec ? launch_tsc_tile<T, false, true>(c, A) : launch_tsc_tile<T, false, false>(c, A));
    if (st != PIC_OK) return st;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->desc.device);
    const int grid = 2 * (sms > 0 ? sms : 152);
    LaunchScope ls(c, KC_LIST_PUSH);
    if (rec) k_tsc_list_push<T, true><<<grid, 256, 0, c->stream>>>(A);
    else k_tsc_list_push<T, false><<<grid, 256, 0, c->stream>>>(A);
    GBPIC_CHECK(c, cudaGetLastError());
    return PIC_OK;
}
template pic_status launch_tsc_push<float>(pic_ctx*, PushArgs<float>&, bool, bool);
template pic_status launch_tsc_push<double>(pic_ctx*, PushArgs<double>&, bool, bool);

template <typename T> pic_status launch_tsc_backpush(pic_ctx* c, PushArgs<T>& A, const T* B0x, const T* B0y, const T* B0z) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->desc.device);
    LaunchScope ls(c, KC_OTHER);
    k_tsc_backpush<T><<<4 * (sms > 0 ? sms : 152), 256, 0, c->stream>>>(A, B0x, B0y, B0z);
    GBPIC_CHECK(c, cudaGetLastError());
    return PIC_OK;
}
template pic_status launch_tsc_backpush<float>(pic_ctx*, PushArgs<float>&, const float*, const float*, const float*);
template pic_status launch_tsc_backpush<double>(pic_ctx*, PushArgs<double>&, const double*, const double*,
                                                const double*);

}  // namespace gbpic

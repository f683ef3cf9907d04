// Internal declarations of the GB300 EM-PIC library: device helpers (inline PTX for
// TMA, mbarrier), the particle arithmetic shared by the tile kernel and the generic
// list kernel, field geometry, and the host-side context.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "gbpic.h"

namespace gbpic {

constexpr int TILE = 8;          // tile edge in cells (8^3 cells per tile)
constexpr int TILE_CELLS = 512;
constexpr int SB = 10;           // staged E/B extent per dim: local cells -1..8
constexpr int SJ = 11;           // shared J extent per dim: local nodes/edges -1..9
constexpr int SJ3 = SJ * SJ * SJ;
constexpr int MAX_WINDOW_PPCX = 64;  // moving window: largest lattice of the new plasma along x
constexpr int MAX_FILTER_PASSES = 8; // current filter: binomial passes per dimension
constexpr int PUSH_WARPS_MAX = 16;   // the tile kernel's CTA has at most 512 threads
constexpr int HOLE = -1;             // cell value of a slot whose particle left the tile last step

// device error bits, OR-ed into Counters::err
enum : int { ERRB_OVERFLOW = 1, ERRB_SUPERLUMINAL = 2, ERRB_NAN = 4, ERRB_TIMEOUT = 8 };

// bounded waits: a try_wait loop gives up after this many polls and raises ERRB_TIMEOUT
constexpr int MBAR_MAX_POLLS = 1 << 24;

template <typename T> struct Prec;
template <> struct Prec<float> {
    // tile kernel CTA: 10 warps and 2 CTAs per SM hold 20 warps at 96 registers; the
    // kernel is latency-bound, so resident warps count for more than registers
    static constexpr int THREADS = 320;
    static constexpr int MINB = 2;
    static constexpr int R = 4;        // consecutive particle slots per lane (one 16-byte load per array)
    static constexpr int BX = 12;      // TMA box inner extent: 12 floats = 48 B (multiple of 16 B)
    static constexpr int JBITS = 40;   // fixed-point fraction bits of a bounded J contribution
};
template <> struct Prec<double> {
    static constexpr int THREADS = 256;
    static constexpr int MINB = 1;
    static constexpr int R = 2;
    static constexpr int BX = 10;      // 10 doubles = 80 B
    static constexpr int JBITS = 50;
};

// Padded Yee field geometry.  Each component array holds local indices -1..n
// per dimension (one ghost layer on each side, periodic images), x fastest,
// with the x pitch padded to a multiple of 8 elements (rows 16-B aligned).
struct Geom {
    int n[3];
    int open_x;       // 1: x is open (absorbing faces); the ghost x = n holds the face nodes
    int nt[3];        // tiles per dimension (ceil(n/8))
    int Px, Gy, Gz;   // x pitch, padded y and z extents (n+2)
    long long N;      // n0 n1 n2
    __host__ __device__ long long pidx(int i, int j, int k) const {
        return ((long long)(k + 1) * Gy + (j + 1)) * Px + (i + 1);
    }
    __host__ __device__ long long cidx(int i, int j, int k) const {   // compact (unpadded)
        return ((long long)k * n[1] + j) * n[0] + i;
    }
    __host__ __device__ long long padded_size() const { return (long long)Px * Gy * Gz; }
    // values of one component in the host layout (an open x line holds n0 + 1 nodes)
    __host__ __device__ long long host_N() const { return (long long)(n[0] + open_x) * n[1] * n[2]; }
};

// Accumulator of the current density J.  FP32 path: 64-bit fixed point (exact,
// order-independent integer atomics in shared memory and HBM).  FP64 path: FP64
// (a fixed unit cannot hold both a relativistic and a cold plasma to 1e-12).
template <typename T> struct JTraits;
template <> struct JTraits<float> {
    using acc_t = long long;
    static constexpr bool fixed = true;
};
template <> struct JTraits<double> {
    using acc_t = double;
    static constexpr bool fixed = false;
};

template <typename T> struct Fields {
    T* E[3];
    T* B[3];
    typename JTraits<T>::acc_t* J[3];   // compact layout
};

// Device counters of one species (double-buffered by step parity).
struct Counters {
    int mover_count[2];
    int spill_count[2];
    int err;
    int escaped;      // particles removed through open x faces
    int pad[2];
};

// One particle outside its tile segment (mover or spill record); cell is global.
template <typename T> struct Rec {
    int cell;
    int id;
    T d[3];
    T u[3];
    T w;
};

template <typename T> struct ParticleArrays {
    int* cell;      // local cell within the owning tile: lx | ly << 3 | lz << 6
    T* d[3];        // in-cell offsets in [0, 1)
    T* u[3];        // u = gamma v
    T* w;
    int* id;        // optional load-order id
    const int* seg_start;
    int* count;     // slots in use: the particles and the holes (cell == HOLE) among them
    const int* cap;
    int* holes;     // holes among the first count slots (the particles that left last step)
};

// ---------------------------------------------------------------------------
// PTX helpers (TMA and mbarrier).

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// 3D tiled TMA load of one box into shared memory, completion counted on bar.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// Particle arithmetic shared by every kernel that pushes.

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float floor_t(float x) { return floorf(x); }
__device__ __forceinline__ double floor_t(double x) { return floor(x); }
// Round-to-nearest-even of |x| < 2^41 to a 64-bit integer with FP32 adds only:
// h = x rounded to a multiple of 2^20 (adding 1.5*2^43 leaves an ulp of 2^20), the
// remainder l = x - h is exact, and both parts become integers by the 1.5*2^23
// mantissa trick.  Equals llrintf(x) without the slower 64-bit conversion path.
__device__ __forceinline__ long long fixed_rn(float x) {
    const float big = 13194139533312.0f;   // 1.5 * 2^43
    const float mag = 12582912.0f;         // 1.5 * 2^23
    const float h = __fsub_rn(__fadd_rn(x, big), big);
    const float l = __fsub_rn(x, h);
    const int hi = __float_as_int(__fadd_rn(__fmul_rn(h, 9.5367431640625e-07f), mag)) - 0x4B400000;  // h / 2^20
    const int lo = __float_as_int(__fadd_rn(l, mag)) - 0x4B400000;
    return ((long long)hi << 20) + (long long)lo;
}
// (a warp sum of 32 bounded terms can leave the window of fixed_rn: convert those
// rare values with the exact 64-bit instruction)
__device__ __forceinline__ long long to_acc(float x) {
    return fabsf(x) < 2199023255552.0f ? fixed_rn(x) : __float2ll_rn(x);   // 2^41
}
__device__ __forceinline__ double to_acc(double x) { return x; }
__device__ __forceinline__ void acc_atomic(long long* p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
}
__device__ __forceinline__ void acc_atomic(double* p, double v) { atomicAdd(p, v); }

// Shared-memory J tile of the tile kernel (element e of NE).  FP32 path: each element
// is a 64-bit fixed-point sum kept as two 32-bit words, lo (bits 0..19 of every term,
// unsigned) at word e and hi (the rest, signed, in units of 2^20) at word NE + e, both
// added with native 32-bit shared reductions (no carry: lo stays below 2^32 for up to
// 4096 terms); the element is hi * 2^20 + lo, an exact integer sum in any order.  The
// value v (fixed-point units as a float) is split exactly: hi = floor(v / 2^20), and
// lo = rint(v - hi * 2^20), an integer in [0, 2^20].  FP64 path: FP64 elements.
__device__ __forceinline__ void tile_add(uint32_t base, int e, int NE, float v) {
    const float hf = floorf(v * 9.5367431640625e-07f);           // v / 2^20
    const int hi = __float2int_rz(hf);
    const unsigned lo = (unsigned)__float2int_rn(__fmaf_rn(hf, -1048576.0f, v));
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(base + 4u * e), "r"(lo) : "memory");
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(base + 4u * (NE + e)), "r"((unsigned)hi) : "memory");
}
__device__ __forceinline__ void tile_add(uint32_t base, int e, int, double v) {
    asm volatile("red.shared.add.f64 [%0], %1;" ::"r"(base + 8u * e), "d"(v) : "memory");
}
__device__ __forceinline__ long long tile_get(const unsigned char* s, int e, int NE, float) {
    const unsigned* w = reinterpret_cast<const unsigned*>(s);
    return ((long long)(int)w[NE + e] << 20) + (long long)w[e];
}
__device__ __forceinline__ double tile_get(const unsigned char* s, int e, int, double) {
    return reinterpret_cast<const double*>(s)[e];
}

// 2 / x: the FP32 path uses the fast approximate division (error ~2 ulp, far inside
// the FP32 tolerance); the FP64 path divides exactly.
__device__ __forceinline__ float two_over(float x) { return __fdividef(2.0f, x); }
__device__ __forceinline__ double two_over(double x) { return 2.0 / x; }

// Staggered CIC weights along one dimension (section 2.5).  A node-located
// component samples cells (i, i+1) with weight s = delta; a half-located one
// samples (i-1, i) or (i, i+1) with s = delta + 1/2 or delta - 1/2.
template <typename T>
__device__ __forceinline__ void half_weight(int i, T delta, int& base, T& s) {
    if (delta >= T(0.5)) {
        base = i;
        s = delta - T(0.5);
    } else {
        base = i - 1;
        s = delta + T(0.5);
    }
}

// Trilinear interpolation of one component from 8 samples fetched by F(x, y, z).
template <typename T, typename Fetch>
__device__ __forceinline__ T trilerp(Fetch F, int bx, int by, int bz, T sx, T sy, T sz) {
    T c00 = F(bx, by, bz) + sx * (F(bx + 1, by, bz) - F(bx, by, bz));
    T c10 = F(bx, by + 1, bz) + sx * (F(bx + 1, by + 1, bz) - F(bx, by + 1, bz));
    T c01 = F(bx, by, bz + 1) + sx * (F(bx + 1, by, bz + 1) - F(bx, by, bz + 1));
    T c11 = F(bx, by + 1, bz + 1) + sx * (F(bx + 1, by + 1, bz + 1) - F(bx, by + 1, bz + 1));
    T c0 = c00 + sy * (c10 - c00);
    T c1 = c01 + sy * (c11 - c01);
    return c0 + sz * (c1 - c0);
}

// Gather E and B (section 2.5) at local cell (x, y, z) + offset (dx, dy, dz);
// F(comp, x, y, z) returns component comp (0..2 = E, 3..5 = B) at a local index.
template <typename T, typename Fetch6>
__device__ __forceinline__ void gather_eb(Fetch6 F, int x, int y, int z, T dx, T dy, T dz, T Ep[3], T Bp[3]) {
    int hx, hy, hz;
    T shx, shy, shz;
    half_weight(x, dx, hx, shx);
    half_weight(y, dy, hy, shy);
    half_weight(z, dz, hz, shz);
    // E: Ex (h,n,n), Ey (n,h,n), Ez (n,n,h);  B: Bx (n,h,h), By (h,n,h), Bz (h,h,n)
    Ep[0] = trilerp<T>([&](int a, int b, int c) { return F(0, a, b, c); }, hx, y, z, shx, dy, dz);
    Ep[1] = trilerp<T>([&](int a, int b, int c) { return F(1, a, b, c); }, x, hy, z, dx, shy, dz);
    Ep[2] = trilerp<T>([&](int a, int b, int c) { return F(2, a, b, c); }, x, y, hz, dx, dy, shz);
    Bp[0] = trilerp<T>([&](int a, int b, int c) { return F(3, a, b, c); }, x, hy, hz, dx, shy, shz);
    Bp[1] = trilerp<T>([&](int a, int b, int c) { return F(4, a, b, c); }, hx, y, hz, shx, dy, shz);
    Bp[2] = trilerp<T>([&](int a, int b, int c) { return F(5, a, b, c); }, hx, hy, z, shx, shy, dz);
}

// Two lanes of arithmetic at once: the FP32 path uses Blackwell's paired FP32
// instructions (one fused multiply-add or add per pair, each element rounded as its
// scalar counterpart), the FP64 path plain scalar pairs.
template <typename T> struct Pair;
template <> struct Pair<float> {
    using t = float2;
    static __device__ __forceinline__ float2 splat(float v) { return make_float2(v, v); }
    static __device__ __forceinline__ float2 make(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
    // b - a, rounded once
    static __device__ __forceinline__ float2 sub(float2 b, float2 a) { return __ffma2_rn(a, make_float2(-1.0f, -1.0f), b); }
};
template <> struct Pair<double> {
    using t = double2;
    static __device__ __forceinline__ double2 splat(double v) { return make_double2(v, v); }
    static __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
    static __device__ __forceinline__ double2 fma(double2 a, double2 b, double2 c) {
        return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y));
    }
    static __device__ __forceinline__ double2 mul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
    static __device__ __forceinline__ double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ double2 sub(double2 b, double2 a) { return make_double2(b.x - a.x, b.y - a.y); }
};

// Relativistic Boris (section 2.4; Boris 1970): u^{n-1/2} -> u^{n+1/2} in place,
// eps = q dt / (2 m).  Returns 1/gamma^{n+1/2}.
template <typename T>
__device__ __forceinline__ T boris(T eps, const T E[3], const T B[3], T u[3]) {
    T um0 = u[0] + eps * E[0], um1 = u[1] + eps * E[1], um2 = u[2] + eps * E[2];
    T ig = rsqrt_t(T(1) + um0 * um0 + um1 * um1 + um2 * um2);
    T t0 = eps * B[0] * ig, t1 = eps * B[1] * ig, t2 = eps * B[2] * ig;
    T f = two_over(T(1) + t0 * t0 + t1 * t1 + t2 * t2);
    T s0 = f * t0, s1 = f * t1, s2 = f * t2;
    T up0 = um0 + (um1 * t2 - um2 * t1);
    T up1 = um1 + (um2 * t0 - um0 * t2);
    T up2 = um2 + (um0 * t1 - um1 * t0);
    u[0] = um0 + (up1 * s2 - up2 * s1) + eps * E[0];
    u[1] = um1 + (up2 * s0 - up0 * s2) + eps * E[1];
    u[2] = um2 + (up0 * s1 - up1 * s0) + eps * E[2];
    return rsqrt_t(T(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
}

// gamma - 1 without cancellation: |u|^2 / (gamma + 1)
template <typename T>
__device__ __forceinline__ T gamma_minus_one(const T u[3]) {
    T u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    T g = T(1) / rsqrt_t(T(1) + u2);
    return u2 / (g + T(1));
}

// Advance one coordinate: offset delta in the current cell moves by disp (cells).
// Returns the cell step (-1, 0, +1, or beyond for a superluminal move) and the
// new offset in [0, 1).  An offset that rounds to 1 goes to 0 of the next cell.
template <typename T>
__device__ __forceinline__ int advance(T delta, T disp, T& out) {
    T x = delta + disp;
    T f = floor_t(x);
    T r = x - f;
    int step = (int)f;
    if (r >= T(1)) {
        r = T(0);
        step += 1;
    }
    out = r;
    return step;
}

// Zigzag relay split of one coordinate (section 2.5, Umeda et al. 2003), written in
// each segment's own cell frame so that the fluxes are exact differences of the
// stored offsets.  Inputs: start offset x1 (cell i1), end offset x2 (cell i1 + s).
// Outputs: segment fluxes F1, F2 (cells) and midpoint offsets W1 (frame i1), W2
// (frame i1 + s).
template <typename T>
__device__ __forceinline__ void relay(T x1, T x2, int s, T& F1, T& F2, T& W1, T& W2) {
    if (s == 0) {                 // relay point at the midpoint
        T D = x2 - x1;
        F1 = T(0.5) * D;
        F2 = F1;
        W1 = x1 + T(0.25) * D;
        W2 = x1 + T(0.75) * D;
    } else if (s > 0) {           // relay point on the upper face of cell i1
        F1 = T(1) - x1;
        F2 = x2;
        W1 = T(0.5) * (x1 + T(1));
        W2 = T(0.5) * x2;
    } else {                      // relay point on the lower face of cell i1
        F1 = -x1;
        F2 = x2 - T(1);
        W1 = T(0.5) * x1;
        W2 = T(0.5) * (x2 + T(1));
    }
}

// Current of one straight segment inside one cell: the 12 edge values
// (units of the fixed-point accumulator).  The product of midpoint weights is
// the zigzag form; the +-F_p F_r / 12 term is the exact flux of a straight
// segment through a trilinear charge cloud, which keeps the deposit exactly
// charge conserving in three dimensions.
//   v[0..3]  Jx at (y+b, z+c), (b,c) = (0,0) (1,0) (0,1) (1,1)
//   v[4..7]  Jy at (x+a, z+c), (a,c) = (0,0) (1,0) (0,1) (1,1)
//   v[8..11] Jz at (x+a, y+b), (a,b) = (0,0) (1,0) (0,1) (1,1)
template <typename T>
__device__ __forceinline__ void segment_values(const T cw[3], const T F[3], const T W[3], T v[12]) {
    const T wx1 = W[0], wy1 = W[1], wz1 = W[2];
    const T wx0 = T(1) - wx1, wy0 = T(1) - wy1, wz0 = T(1) - wz1;
    const T twelfth = T(1) / T(12);
    T ax = cw[0] * F[0], ay = cw[1] * F[1], az = cw[2] * F[2];
    T kx = F[1] * F[2] * twelfth, ky = F[0] * F[2] * twelfth, kz = F[0] * F[1] * twelfth;
    v[0] = ax * (wy0 * wz0 + kx);
    v[1] = ax * (wy1 * wz0 - kx);
    v[2] = ax * (wy0 * wz1 - kx);
    v[3] = ax * (wy1 * wz1 + kx);
    v[4] = ay * (wx0 * wz0 + ky);
    v[5] = ay * (wx1 * wz0 - ky);
    v[6] = ay * (wx0 * wz1 - ky);
    v[7] = ay * (wx1 * wz1 + ky);
    v[8] = az * (wx0 * wy0 + kz);
    v[9] = az * (wx1 * wy0 - kz);
    v[10] = az * (wx0 * wy1 - kz);
    v[11] = az * (wx1 * wy1 + kz);
}

// segment_values as six pairs (v[0], v[1]), (v[2], v[3]), ... of the same values.
template <typename T>
__device__ __forceinline__ void segment_values_pairs(const T cw[3], const T F[3], const T W[3],
                                                     typename Pair<T>::t v[6]) {
    using PT = Pair<T>;
    using P2 = typename PT::t;
    const T twelfth = T(1) / T(12);
    const T kx = F[1] * F[2] * twelfth, ky = F[0] * F[2] * twelfth, kz = F[0] * F[1] * twelfth;
    const P2 wx = PT::make(T(1) - W[0], W[0]), wy = PT::make(T(1) - W[1], W[1]);
    const T wz0 = T(1) - W[2], wz1 = W[2], wy0 = T(1) - W[1], wy1 = W[1];
    const P2 ax = PT::splat(cw[0] * F[0]), ay = PT::splat(cw[1] * F[1]), az = PT::splat(cw[2] * F[2]);
    v[0] = PT::mul(ax, PT::fma(wy, PT::splat(wz0), PT::make(kx, -kx)));
    v[1] = PT::mul(ax, PT::fma(wy, PT::splat(wz1), PT::make(-kx, kx)));
    v[2] = PT::mul(ay, PT::fma(wx, PT::splat(wz0), PT::make(ky, -ky)));
    v[3] = PT::mul(ay, PT::fma(wx, PT::splat(wz1), PT::make(-ky, ky)));
    v[4] = PT::mul(az, PT::fma(wx, PT::splat(wy0), PT::make(kz, -kz)));
    v[5] = PT::mul(az, PT::fma(wx, PT::splat(wy1), PT::make(-kz, kz)));
}

// Scatter 12 segment values of the cell (x, y, z) through Add(comp, x, y, z, fixed).
template <typename T, typename AddFn>
__device__ __forceinline__ void scatter12(AddFn Add, int x, int y, int z, const T v[12]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int b = q & 1, c = q >> 1;
        Add(0, x, y + b, z + c, to_acc(v[q]));
        Add(1, x + b, y, z + c, to_acc(v[4 + q]));
        Add(2, x + b, y + c, z, to_acc(v[8 + q]));
    }
}

// Edge (component, local x, y, z) of slot s (0..11) of the cell (x, y, z), in the
// order of segment_values.
__device__ __forceinline__ void slot_edge(int s, int x, int y, int z, int& comp, int& ex, int& ey, int& ez) {
    comp = s >> 2;
    const int q = s & 3, b = q & 1, c = q >> 1;
    ex = x + (comp == 0 ? 0 : b);
    ey = y + (comp == 0 ? b : comp == 1 ? 0 : c);
    ez = z + (comp == 2 ? 0 : c);
}

// Whole zigzag deposit of one move (section 2.5): start cell (x, y, z) offsets d1,
// cell steps s[3], end offsets d2; cw = q w / (dt d_p d_r) in fixed-point units.
template <typename T, typename AddFn>
__device__ __forceinline__ void zigzag_deposit(AddFn Add, int x, int y, int z, const T d1[3], const int s[3],
                                               const T d2[3], const T cw[3]) {
    T F1[3], F2[3], W1[3], W2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) relay(d1[k], d2[k], s[k], F1[k], F2[k], W1[k], W2[k]);
    T v[12];
    segment_values(cw, F1, W1, v);
    if ((s[0] | s[1] | s[2]) == 0) {
        T v2[12];
        segment_values(cw, F2, W2, v2);
#pragma unroll
        for (int q = 0; q < 12; ++q) v[q] += v2[q];
        scatter12(Add, x, y, z, v);
    } else {
        scatter12(Add, x, y, z, v);
        segment_values(cw, F2, W2, v);
        scatter12(Add, x + s[0], y + s[1], z + s[2], v);
    }
}

// Esirkepov's charge-conserving deposit (Esirkepov 2001; section 2.5 names it next to
// ZigZag) with the CIC shape, for a move from offsets d1 in cell (x, y, z) to offsets d2
// in cell (x, y, z) + s.  Per dimension the support is the nodes b .. b + 2, b = min(0, s)
// (relative to the start cell), with S0, S1 the node weights before and after and
// DS = S1 - S0;  Wx = DSx (S0y S0z + DSy S0z / 2 + S0y DSz / 2 + DSy DSz / 3) (y, z
// cyclically) and Jx at the edge b + i + 1/2 is -cw_x times the sum of Wx over the
// nodes b .. b + i.  esk_value returns one of the 54 values (component comp, edge i of
// 2, nodes jp, jr of 3 along the two other dimensions in cyclic order); X1, X2 are the
// positions relative to the support's first node.
template <typename T> __device__ __forceinline__ T cic_w(T r) {
    r = r < T(0) ? -r : r;
    return r < T(1) ? T(1) - r : T(0);
}
// element k of a 3-vector by selects (a runtime index into a local array would put the
// array in local memory)
template <typename T> __device__ __forceinline__ T sel3(const T a[3], int k) {
    return k == 0 ? a[0] : (k == 1 ? a[1] : a[2]);
}
template <typename T>
__device__ __forceinline__ T esk_value(const T X1[3], const T X2[3], const T cw[3], int comp, int i, int jp, int jr) {
    const int p = comp == 2 ? 0 : comp + 1, r = comp == 0 ? 2 : comp - 1;
    const T x1p = sel3(X1, p), x2p = sel3(X2, p), x1r = sel3(X1, r), x2r = sel3(X2, r);
    const T x1c = sel3(X1, comp), x2c = sel3(X2, comp);
    const T s0p = cic_w(x1p - T(jp)), dsp = cic_w(x2p - T(jp)) - s0p;
    const T s0r = cic_w(x1r - T(jr)), dsr = cic_w(x2r - T(jr)) - s0r;
    const T t = s0p * s0r + T(0.5) * dsp * s0r + T(0.5) * s0p * dsr + dsp * dsr * T(1.0 / 3.0);
    T acc = (cic_w(x2c) - cic_w(x1c)) * t;
    if (i == 1) acc += (cic_w(x2c - T(1)) - cic_w(x1c - T(1))) * t;
    return -sel3(cw, comp) * acc;
}

// The whole Esirkepov deposit of one move through Add(comp, x, y, z, fixed) (global
// or tile coordinates of the J component's location).
template <typename T, typename AddFn>
__device__ __forceinline__ void esirkepov_deposit(AddFn Add, int x, int y, int z, const T d1[3], const int s[3],
                                                  const T d2[3], const T cw[3]) {
    int b[3];
    T X1[3], X2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        b[k] = s[k] < 0 ? -1 : 0;
        X1[k] = d1[k] - T(b[k]);
        X2[k] = d2[k] + T(s[k] - b[k]);
    }
    const int o[3] = {x + b[0], y + b[1], z + b[2]};
    for (int comp = 0; comp < 3; ++comp) {
        const int p = comp == 2 ? 0 : comp + 1, r = comp == 0 ? 2 : comp - 1;
        for (int i = 0; i < 2; ++i)
            for (int jp = 0; jp < 3; ++jp)
                for (int jr = 0; jr < 3; ++jr) {
                    const T v = esk_value(X1, X2, cw, comp, i, jp, jr);
                    if (v == T(0)) continue;
                    int c3[3];
                    c3[comp] = o[comp] + i;
                    c3[p] = o[p] + jp;
                    c3[r] = o[r] + jr;
                    Add(comp, c3[0], c3[1], c3[2], to_acc(v));
                }
    }
}

// Running maximum of non-negative values that lets a non-finite value through as +inf
// (fmax alone returns the other operand of a NaN, which would hide a run that blew up).
__device__ __forceinline__ double max_nf(double m, double v) { return isfinite(v) ? fmax(m, v) : HUGE_VAL; }

__device__ __forceinline__ int wrap_idx(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Periodic wrap of an index at most one period outside [0, n) (-n <= i < 2n): a cell
// index after a move of at most one cell, without a division.
__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
// The same for -n <= i < 3n (an edge next to a moved cell on a grid of one cell or more).
__device__ __forceinline__ int wrap2(int i, int n) {
    i = i < 0 ? i + n : i;
    i = i >= n ? i - n : i;
    return i >= n ? i - n : i;
}

// Ghost images of interior index i along a periodic dimension of n cells.
__device__ __forceinline__ int images(int i, int n, int out[3]) {
    int m = 0;
    out[m++] = i;
    if (i == 0) out[m++] = n;
    if (i == n - 1) out[m++] = -1;
    return m;
}

// Store v0..v2 at (i, j, k) and at its periodic ghost images.  An open x has no x
// images (its ghost x = -1 stays zero and x = n holds the face nodes), and i may then
// be n itself.
template <typename T>
__device__ __forceinline__ void store3(const Geom& g, T* a0, T* a1, T* a2, int i, int j, int k, T v0, T v1, T v2) {
    const long long c = g.pidx(i, j, k);
    a0[c] = v0;
    a1[c] = v1;
    a2[c] = v2;
    const bool edge = (!g.open_x && (i == 0 || i == g.n[0] - 1)) || j == 0 || j == g.n[1] - 1 || k == 0 ||
                      k == g.n[2] - 1;
    if (!edge) return;
    int xs[3], ys[3], zs[3];
    int nx = 1;
    xs[0] = i;
    if (!g.open_x) nx = images(i, g.n[0], xs);
    const int ny = images(j, g.n[1], ys), nz = images(k, g.n[2], zs);
    for (int c3 = 0; c3 < nz; ++c3)
        for (int b = 0; b < ny; ++b)
            for (int a = 0; a < nx; ++a) {
                if (a == 0 && b == 0 && c3 == 0) continue;
                const long long q = g.pidx(xs[a], ys[b], zs[c3]);
                a0[q] = v0;
                a1[q] = v1;
                a2[q] = v2;
            }
}

// One component at (i, j, k) with its y and z images (face planes of an open x).
template <typename T>
__device__ __forceinline__ void store1_yz(const Geom& g, T* a, int i, int j, int k, T v) {
    int ys[3], zs[3];
    const int ny = images(j, g.n[1], ys), nz = images(k, g.n[2], zs);
    for (int c3 = 0; c3 < nz; ++c3)
        for (int b = 0; b < ny; ++b) a[g.pidx(i, ys[b], zs[c3])] = v;
}

// x index of a global cell after a move: wrapped (periodic) or -1 when it left an open x.
__device__ __forceinline__ int x_after(const Geom& g, int gx) {
    if (g.open_x) return (gx < 0 || gx >= g.n[0]) ? -1 : gx;
    return wrap_idx(gx, g.n[0]);
}
// The same for a global x at most one cell outside the box (-1 <= gx <= n).
__device__ __forceinline__ int x_after1(const Geom& g, int gx) {
    if (g.open_x) return (gx < 0 || gx >= g.n[0]) ? -1 : gx;
    return wrap1(gx, g.n[0]);
}

// ---------------------------------------------------------------------------
// Host side.

enum KernelClass { KC_FARADAY = 0, KC_TILE_PUSH, KC_LIST_PUSH, KC_APPEND, KC_AMPERE, KC_SORT, KC_OTHER, KC_ESK, KC_COUNT };

struct SpeciesDev {
    double q = 0, m = 0;
    int64_t n_loaded = 0;
    int64_t cap_total = 0;
    void* base[2] = {nullptr, nullptr};   // SoA blocks: current and sort target (ping-pong)
    ParticleArrays<float> pf[2] = {};     // valid when FP32
    ParticleArrays<double> pd[2] = {};    // valid when FP64
    int cur = 0;                          // which block holds the particles
    size_t pbytes = 0;                    // bytes of one SoA block
    int* seg_start = nullptr;
    int* count = nullptr;
    int* cap = nullptr;
    int* holes = nullptr;
    int* hist[2] = {nullptr, nullptr};    // per tile and block: particles per cell (TILE_CELLS ints)
    int* split_buf = nullptr;             // split tiles: output ranges (TILE_CELLS per tile), input counts
    void* esk_buf = nullptr;              // Esirkepov's deposit: exported crosser records (push.cu)
    int* esk_cnt = nullptr;               // their counts per tile and warp
    int esk_wcap = 0;                     // records per tile and warp
    void* movers = nullptr;
    int mover_cap = 0;
    void* spill = nullptr;
    int spill_cap = 0;
    Counters* ctr = nullptr;
    double jscale = 0;               // physical J per fixed-point unit from this species
    int64_t n_injected = 0;          // particles a moving window has added (ids from n_loaded on)
    std::vector<int> h_seg_start, h_cap;
};

template <typename T> inline ParticleArrays<T>& arrays(SpeciesDev& s);
template <> inline ParticleArrays<float>& arrays<float>(SpeciesDev& s) { return s.pf[s.cur]; }
template <> inline ParticleArrays<double>& arrays<double>(SpeciesDev& s) { return s.pd[s.cur]; }
template <typename T> inline ParticleArrays<T>& arrays_alt(SpeciesDev& s);
template <> inline ParticleArrays<float>& arrays_alt<float>(SpeciesDev& s) { return s.pf[s.cur ^ 1]; }
template <> inline ParticleArrays<double>& arrays_alt<double>(SpeciesDev& s) { return s.pd[s.cur ^ 1]; }

struct TimingPair {
    int cls;
    cudaEvent_t a, b;
};

}  // namespace gbpic

struct pic_ctx {
    pic_grid_desc desc{};
    gbpic::Geom g{};
    int prec = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t esize = 4;
    void* E[3] = {};
    void* B[3] = {};
    void* J[3] = {};          // JTraits<T>::acc_t arrays, compact layout
    double jscale = 0;        // physical J per fixed-point unit (shared by all species)
    double jinv = 0;          // 1 / jscale
    double jscale_J = 1.0;    // the unit of the J the last cycle kept (jscale then)
    bool fields_set = false;
    bool j_dirty = false;     // J holds the last deposit and must be cleared before stepping
    int64_t step = 0;
    std::vector<gbpic::SpeciesDev> species;
    CUtensorMap tmap[6];
    // diagnostics
    double* rho = nullptr;
    double* rho_prev = nullptr;
    double* gref = nullptr;
    bool gref_valid = false;
    int64_t rho_prev_step = -1;
    double* dacc = nullptr;   // device accumulators for reductions
    double* hist = nullptr;
    int hist_cap = 0;
    int64_t hist_written = 0;
    // bookkeeping
    int64_t launches = 0;
    bool timing = false;
    std::vector<gbpic::TimingPair> pending;
    std::vector<cudaEvent_t> event_pool;
    double kc_ms[gbpic::KC_COUNT] = {};
    int64_t kc_n[gbpic::KC_COUNT] = {};
    std::vector<void*> allocations;
    std::string err;
    void* adj = nullptr;      // checkpointed adjoint state (adjoint.cu)
    // open x: the laser sheet and the Mur buffer (Ey, Ez of planes 0, 1, n-1, n)
    bool laser_on = false;
    pic_laser_desc laser{};
    void* mur_old = nullptr;
    // moving window (open x)
    bool window_on = false;
    pic_window_desc window{};
    int64_t window_moves = 0;
    int64_t window_moves_at_rho = -1;   // window_moves when rho_prev was taken
    int64_t window_moves_at_gref = 0;   // window_moves when the Gauss reference was taken
    // compensated binomial current filter (0 passes: off)
    int filter_passes = 0;
    int filter_compensate = 0;
    int filter_h = 0;                   // half width of the per-dimension kernel
    double filter_K[2 * gbpic::MAX_FILTER_PASSES + 3] = {};
    void* Jtmp[3] = {};                 // second J set (the filter ping-pongs)
    // perfectly conducting wall planes (y = 0, z = 0) and the port on the face x = 0
    int pec_y = 0, pec_z = 0;
    bool port_on = false;
    pic_port_desc port{};
    int deposit = 0;                    // pic_deposit: ZigZag or Esirkepov
    int shape = 1;                      // pic_shape: CIC (1) or quadratic TSC (2)
    int wait_polls = -1;                // tile kernel staging wait limit (negative: MBAR_MAX_POLLS)
    cudaGraphExec_t step_graph = nullptr;   // the last two-cycle graph of pic_step (api.cu)
    cudaStream_t capture_stream = nullptr;  // the stream that graph is captured on
};

namespace gbpic {

// launchers (defined in the .cu files)
pic_status launch_faraday_half(pic_ctx* c, double* rec);
pic_status launch_ampere(pic_ctx* c, bool zero_j);
pic_status launch_push_species(pic_ctx* c, SpeciesDev& s, int parity, double* krec, int xshift, bool inject);
pic_status launch_window_shift(pic_ctx* c);
pic_status launch_current_filter(pic_ctx* c);
pic_status launch_guide(pic_ctx* c);
bool window_moves_after(const pic_ctx* c, int64_t step);
pic_status launch_backpush(pic_ctx* c, SpeciesDev& s);
template <typename T> pic_status curl_to_b(pic_ctx* c, T* const E[3], T* const B[3], double coef);
template <typename T> pic_status curl_to_e(pic_ctx* c, T* const E[3], T* const B[3], double coef);
pic_status step_once(pic_ctx* c, double* rec, bool keep_j);
void update_jscale(pic_ctx* c);
void adjoint_free(pic_ctx* c);
pic_status energy_sums(pic_ctx* c, double* UE, double* UB);
pic_status launch_open_x_before_ampere(pic_ctx* c);
pic_status launch_open_x_after_ampere(pic_ctx* c);
pic_status load_species_impl(pic_ctx* c, const pic_species_desc* d, SpeciesDev& s);
pic_status get_particles_impl(pic_ctx* c, SpeciesDev& s, double* out_dev, int64_t n_out);
pic_status pack_fields(pic_ctx* c, double* E, double* B, double* J);   // device outputs
pic_status unpack_fields(pic_ctx* c, const double* E, const double* B); // device inputs
pic_status diagnostics_impl(pic_ctx* c, pic_diag* out);
pic_status make_tensor_maps(pic_ctx* c);
pic_status static_scratch_prepare(pic_ctx* c);   // static_check.cu

// helpers (api.cu)
void* dev_alloc(pic_ctx* c, size_t bytes);
// Raises kernel kern's dynamic shared-memory limit to bytes on device dev, once per
// (kernel, device, size): cudaFuncSetAttribute acts on the calling thread's current
// device only.
cudaError_t raise_smem_limit(const void* kern, size_t bytes, int dev);
void dev_free(pic_ctx* c, void* p);
pic_status cuda_fail(pic_ctx* c, cudaError_t e, const char* what);
void timing_begin(pic_ctx* c, int cls, cudaEvent_t* a);
void timing_end(pic_ctx* c, int cls, cudaEvent_t a);
int64_t count_alive(pic_ctx* c, SpeciesDev& s, int64_t* spilled);
pic_status reserve_esk_records(pic_ctx* c, SpeciesDev& s);
// Captures the work that body enqueues on c->stream as a CUDA graph (on a stream of the
// context's own: the legacy default stream cannot be captured) and launches it once on
// c->stream.  *done is false when the capture or instantiation failed and nothing was
// launched; body's host-side effects then remain for the caller to undo.
pic_status run_as_graph(pic_ctx* c, const std::function<pic_status()>& body, bool* done);

#define GBPIC_CHECK(c, call)                                              \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return ::gbpic::cuda_fail((c), e_, #call); \
    } while (0)

// Makes a device current for one entry point and gives the caller's current device
// back when the entry point returns, so that a host program driving several devices
// keeps the device it had selected.
struct DeviceScope {
    int prev = -1;
    bool ok = true;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceScope() {
        if (prev >= 0) {
            int cur = -1;
            if (cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
        }
    }
    DeviceScope(const DeviceScope&) = delete;
    DeviceScope& operator=(const DeviceScope&) = delete;
};

// Bracket one launch with optional timing events and count it.
struct LaunchScope {
    pic_ctx* c;
    int cls;
    cudaEvent_t a = nullptr;
    LaunchScope(pic_ctx* c_, int cls_) : c(c_), cls(cls_) {
        timing_begin(c, cls, &a);
        c->launches++;
    }
    ~LaunchScope() { timing_end(c, cls, a); }
};

}  // namespace gbpic

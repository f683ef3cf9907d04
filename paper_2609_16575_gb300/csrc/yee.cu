// Yee FDTD curl updates (KEMPIC-3D section 2.3):
//   k_faraday_half   B <- B - (dt/2) curl E          (Eq. (13) and cyclic permutations)
//   k_ampere         E <- E + dt (curl B - J); J <- 0  (Eq. (14) and cyclic permutations)
// One thread per cell, x fastest (coalesced rows).  Each kernel writes the value of
// an edge cell also into its periodic ghost images (local -1 and n), so the next
// stencil and the tile kernel's TMA staging read valid ghosts without a separate
// halo pass.
#include <cmath>

#include <algorithm>
#include "pic_internal.cuh"

namespace gbpic {

template <typename T> struct YeeArgs {
    Geom g;
    Fields<T> f;
    T cx, cy, cz;   // frac * dt / d
    T dt;           // Ampere: dt
    T jscale;       // physical J per fixed-point unit
    int zero_j;
    int has_j;      // 0: curl update only (adjoint fields)
    double* rec;    // optional: rec[0] += 1/2 dV sum E^2, rec[1] += 1/2 dV sum B_new^2
    double half_dv;
};

__device__ __forceinline__ void block_add2(double a, double b, double* dst) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    __shared__ double ra[32], rb[32];
    const int t = threadIdx.x + threadIdx.y * blockDim.x;
    const int nw = (blockDim.x * blockDim.y + 31) / 32;
    if ((t & 31) == 0) {
        ra[t >> 5] = a;
        rb[t >> 5] = b;
    }
    __syncthreads();
    if (t == 0) {
        double sa = 0, sb = 0;
        for (int w = 0; w < nw; ++w) {
            sa += ra[w];
            sb += rb[w];
        }
        atomicAdd(dst, sa);
        atomicAdd(dst + 1, sb);
    }
}

template <typename T, bool REC>
__global__ void __launch_bounds__(256) k_faraday_half(YeeArgs<T> A) {
    const Geom& g = A.g;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    double se = 0, sb = 0;
    if (i < g.n[0] && j < g.n[1]) {
        const long long c = g.pidx(i, j, k);
        const long long sy = g.Px, sz = (long long)g.Px * g.Gy;
        const T* Ex = A.f.E[0];
        const T* Ey = A.f.E[1];
        const T* Ez = A.f.E[2];
        const T ex = Ex[c], ey = Ey[c], ez = Ez[c];
        // Bx(i, j+1/2, k+1/2) -= dt/dy [Ez(j+1) - Ez(j)] - dt/dz [Ey(k+1) - Ey(k)]
        const T bx = A.f.B[0][c] - (A.cy * (Ez[c + sy] - ez) - A.cz * (Ey[c + sz] - ey));
        // By(i+1/2, j, k+1/2) -= dt/dz [Ex(k+1) - Ex(k)] - dt/dx [Ez(i+1) - Ez(i)]
        const T by = A.f.B[1][c] - (A.cz * (Ex[c + sz] - ex) - A.cx * (Ez[c + 1] - ez));
        // Bz(i+1/2, j+1/2, k) -= dt/dx [Ey(i+1) - Ey(i)] - dt/dy [Ex(j+1) - Ex(j)]
        const T bz = A.f.B[2][c] - (A.cx * (Ey[c + 1] - ey) - A.cy * (Ex[c + sy] - ex));
        store3(g, A.f.B[0], A.f.B[1], A.f.B[2], i, j, k, bx, by, bz);
        if (REC) {
            se = (double)ex * ex + (double)ey * ey + (double)ez * ez;
            sb = (double)bx * bx + (double)by * by + (double)bz * bz;
        }
        if (g.open_x && i == g.n[0] - 1) {
            // the face x = n of an open x carries Bx (and Ey, Ez set by the Mur condition)
            const long long f = g.pidx(i + 1, j, k);
            const T eyf = Ey[f], ezf = Ez[f];
            const T bxf = A.f.B[0][f] - (A.cy * (Ez[f + sy] - ezf) - A.cz * (Ey[f + sz] - eyf));
            store1_yz(g, A.f.B[0], i + 1, j, k, bxf);
            if (REC) {
                se += (double)eyf * eyf + (double)ezf * ezf;
                sb += (double)bxf * bxf;
            }
        }
    }
    if (REC) block_add2(se * A.half_dv, sb * A.half_dv, A.rec);
}

// J in the working precision: fixed point times its unit (FP32), or FP64 as stored.
__device__ __forceinline__ float j_value(long long v, float s) { return __ll2float_rn(v) * s; }
__device__ __forceinline__ double j_value(double v, double) { return v; }

template <typename T>
__global__ void __launch_bounds__(256) k_ampere(YeeArgs<T> A) {
    const Geom& g = A.g;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.n[0] || j >= g.n[1]) return;
    const long long c = g.pidx(i, j, k);
    const long long cj = g.cidx(i, j, k);
    const long long sy = g.Px, sz = (long long)g.Px * g.Gy;
    const T* Bx = A.f.B[0];
    const T* By = A.f.B[1];
    const T* Bz = A.f.B[2];
    const T bx = Bx[c], by = By[c], bz = Bz[c];
    using Acc = typename JTraits<T>::acc_t;
    const Acc jx = A.has_j ? A.f.J[0][cj] : Acc(0), jy = A.has_j ? A.f.J[1][cj] : Acc(0),
              jz = A.has_j ? A.f.J[2][cj] : Acc(0);
    if (A.has_j && A.zero_j) {
        A.f.J[0][cj] = Acc(0);
        A.f.J[1][cj] = Acc(0);
        A.f.J[2][cj] = Acc(0);
    }
    // Ex(i+1/2, j, k) += dt/dy [Bz(j+1/2) - Bz(j-1/2)] - dt/dz [By(k+1/2) - By(k-1/2)] - dt Jx
    const T ex = A.f.E[0][c] + (A.cy * (bz - Bz[c - sy]) - A.cz * (by - By[c - sz])) - A.dt * j_value(jx, A.jscale);
    // Ey(i, j+1/2, k) += dt/dz [Bx(k+1/2) - Bx(k-1/2)] - dt/dx [Bz(i+1/2) - Bz(i-1/2)] - dt Jy
    T ey = A.f.E[1][c] + (A.cz * (bx - Bx[c - sz]) - A.cx * (bz - Bz[c - 1])) - A.dt * j_value(jy, A.jscale);
    // Ez(i, j, k+1/2) += dt/dx [By(i+1/2) - By(i-1/2)] - dt/dy [Bx(j+1/2) - Bx(j-1/2)] - dt Jz
    T ez = A.f.E[2][c] + (A.cx * (by - By[c - 1]) - A.cy * (bx - Bx[c - sy])) - A.dt * j_value(jz, A.jscale);
    if (g.open_x && i == 0) {   // the face x = 0 of an open x follows the Mur condition instead
        ey = A.f.E[1][c];
        ez = A.f.E[2][c];
    }
    store3(g, A.f.E[0], A.f.E[1], A.f.E[2], i, j, k, ex, ey, ez);
}

template <typename T>
static YeeArgs<T> yee_args(pic_ctx* c, double frac) {
    YeeArgs<T> A{};
    A.g = c->g;
    for (int k = 0; k < 3; ++k) {
        A.f.E[k] = static_cast<T*>(c->E[k]);
        A.f.B[k] = static_cast<T*>(c->B[k]);
        A.f.J[k] = static_cast<typename JTraits<T>::acc_t*>(c->J[k]);
    }
    const double dt = c->desc.dt;
    A.cx = (T)(frac * dt / c->desc.d[0]);
    A.cy = (T)(frac * dt / c->desc.d[1]);
    A.cz = (T)(frac * dt / c->desc.d[2]);
    A.dt = (T)dt;
    A.jscale = (T)c->jscale;
    A.half_dv = 0.5 * c->desc.d[0] * c->desc.d[1] * c->desc.d[2];
    return A;
}

static dim3 yee_grid(const Geom& g) { return dim3((g.n[0] + 31) / 32, (g.n[1] + 7) / 8, g.n[2]); }

template <typename T>
static pic_status faraday_t(pic_ctx* c, double* rec) {
    YeeArgs<T> A = yee_args<T>(c, 0.5);
    A.rec = rec;
    LaunchScope ls(c, KC_FARADAY);
    if (rec) k_faraday_half<T, true><<<yee_grid(c->g), dim3(32, 8), 0, c->stream>>>(A);
    else k_faraday_half<T, false><<<yee_grid(c->g), dim3(32, 8), 0, c->stream>>>(A);
    GBPIC_CHECK(c, cudaGetLastError());
    return PIC_OK;
}

template <typename T>
static pic_status ampere_t(pic_ctx* c, bool zero_j) {
    YeeArgs<T> A = yee_args<T>(c, 1.0);
    A.zero_j = zero_j ? 1 : 0;
    A.has_j = 1;
    LaunchScope ls(c, KC_AMPERE);
    k_ampere<T><<<yee_grid(c->g), dim3(32, 8), 0, c->stream>>>(A);
    GBPIC_CHECK(c, cudaGetLastError());
    return PIC_OK;
}

pic_status launch_faraday_half(pic_ctx* c, double* rec) {
    return c->prec == PIC_FP64 ? faraday_t<double>(c, rec) : faraday_t<float>(c, rec);
}

pic_status launch_ampere(pic_ctx* c, bool zero_j) {
    return c->prec == PIC_FP64 ? ampere_t<double>(c, zero_j) : ampere_t<float>(c, zero_j);
}

// Curl updates on arbitrary arrays (the adjoint fields): B <- B - coef curl E on the
// Faraday stencil, and E <- E + coef curl B on the Ampere stencil, with ghost images.
template <typename T>
pic_status curl_to_b(pic_ctx* c, T* const E[3], T* const B[3], double coef) {
    YeeArgs<T> A{};
    A.g = c->g;
    for (int k = 0; k < 3; ++k) {
        A.f.E[k] = E[k];
        A.f.B[k] = B[k];
    }
    A.cx = (T)(coef / c->desc.d[0]);
    A.cy = (T)(coef / c->desc.d[1]);
    A.cz = (T)(coef / c->desc.d[2]);
    LaunchScope ls(c, KC_OTHER);
    k_faraday_half<T, false><<<yee_grid(c->g), dim3(32, 8), 0, c->stream>>>(A);
    GBPIC_CHECK(c, cudaGetLastError());
    return PIC_OK;
}

template <typename T>
pic_status curl_to_e(pic_ctx* c, T* const E[3], T* const B[3], double coef) {
    YeeArgs<T> A{};
    A.g = c->g;
    for (int k = 0; k < 3; ++k) {
        A.f.E[k] = E[k];
        A.f.B[k] = B[k];
    }
    A.cx = (T)(coef / c->desc.d[0]);
    A.cy = (T)(coef / c->desc.d[1]);
    A.cz = (T)(coef / c->desc.d[2]);
    A.has_j = 0;
    LaunchScope ls(c, KC_OTHER);
    k_ampere<T><<<yee_grid(c->g), dim3(32, 8), 0, c->stream>>>(A);
    GBPIC_CHECK(c, cudaGetLastError());
    return PIC_OK;
}

template pic_status curl_to_b<float>(pic_ctx*, float* const*, float* const*, double);
template pic_status curl_to_b<double>(pic_ctx*, double* const*, double* const*, double);
template pic_status curl_to_e<double>(pic_ctx*, double* const*, double* const*, double);

// ---------------------------------------------------------------------------
// Open x (boundary and external-source modules of section 2.6; section 4 set-up).

// Ey, Ez of the planes x = 0, 1, n-1, n before the Ampere update: old[comp][plane][k][j].
template <typename T>
__global__ void k_mur_save(Geom g, const T* Ey, const T* Ez, T* old) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (j >= g.n[1]) return;
    const long long P = (long long)g.n[1] * g.n[2], p = (long long)k * g.n[1] + j;
    const int planes[4] = {0, 1, g.n[0] - 1, g.n[0]};
    for (int q = 0; q < 4; ++q) {
        old[q * P + p] = Ey[g.pidx(planes[q], j, k)];
        old[(4 + q) * P + p] = Ez[g.pidx(planes[q], j, k)];
    }
}

// First-order Mur on the two faces: E^{n+1}(0) = E^n(1) + kk (E^{n+1}(1) - E^n(0)),
// E^{n+1}(n) = E^n(n-1) + kk (E^{n+1}(n-1) - E^n(n)), kk = (dt - dx) / (dt + dx).
template <typename T>
__global__ void k_mur_apply(Geom g, T* Ey, T* Ez, const T* old, T kk) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (j >= g.n[1]) return;
    const long long P = (long long)g.n[1] * g.n[2], p = (long long)k * g.n[1] + j;
    const int n = g.n[0];
    T* F[2] = {Ey, Ez};
    for (int c = 0; c < 2; ++c) {
        const T* o = old + (long long)c * 4 * P;
        const T e0 = o[1 * P + p] + kk * (F[c][g.pidx(1, j, k)] - o[0 * P + p]);
        const T en = o[2 * P + p] + kk * (F[c][g.pidx(n - 1, j, k)] - o[3 * P + p]);
        store1_yz(g, F[c], 0, j, k, e0);
        store1_yz(g, F[c], n, j, k, en);
    }
}

// Laser sheet: J_y(plane, j, k) += -2 a exp(-r^2 / w0^2) / dx (a = a(t) from the host).
__device__ __forceinline__ void j_add(long long* J, long long e, double v, double jinv) { J[e] += __double2ll_rn(v * jinv); }
__device__ __forceinline__ void j_add(double* J, long long e, double v, double) { J[e] += v; }

template <typename A>
__global__ void k_laser(Geom g, A* Jy, int plane, double amp, double w0, double yc, double zc, double dx, double dy,
                        double dz, double jinv) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (j >= g.n[1]) return;
    const double y = (j + 0.5) * dy - yc, z = k * dz - zc;
    j_add(Jy, g.cidx(plane, j, k), -2.0 * amp * exp(-(y * y + z * z) / (w0 * w0)) / dx, jinv);
}

template <typename T>
static pic_status open_before_t(pic_ctx* c) {
    const Geom& g = c->g;
    dim3 grid((g.n[1] + 127) / 128, g.n[2]);
    if (c->laser_on) {
        const pic_laser_desc& L = c->laser;
        const double t = (c->step + 0.5) * c->desc.dt, s = t - L.t_peak;
        const double amp = L.a0 * std::exp(-2.0 * std::log(2.0) * s * s / (L.tau * L.tau)) * std::sin(L.omega * s);
        const double* d = c->desc.d;
        LaunchScope ls(c, KC_OTHER);
        using Acc = typename JTraits<T>::acc_t;
        k_laser<Acc><<<grid, 128, 0, c->stream>>>(g, static_cast<Acc*>(c->J[1]), L.plane, amp, L.w0, L.yc * d[1],
                                                   L.zc * d[2], d[0], d[1], d[2], c->jinv);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    LaunchScope ls(c, KC_OTHER);
    k_mur_save<T><<<grid, 128, 0, c->stream>>>(g, (const T*)c->E[1], (const T*)c->E[2], (T*)c->mur_old);
    GBPIC_CHECK(c, cudaGetLastError());
    return PIC_OK;
}

template <typename T>
static pic_status open_after_t(pic_ctx* c) {
    const Geom& g = c->g;
    dim3 grid((g.n[1] + 127) / 128, g.n[2]);
    const double kk = (c->desc.dt - c->desc.d[0]) / (c->desc.dt + c->desc.d[0]);
    LaunchScope ls(c, KC_OTHER);
    k_mur_apply<T><<<grid, 128, 0, c->stream>>>(g, (T*)c->E[1], (T*)c->E[2], (const T*)c->mur_old, (T)kk);
    GBPIC_CHECK(c, cudaGetLastError());
    return PIC_OK;
}

// ---------------------------------------------------------------------------
// Moving window (section 2.2: an operation at the end of the cycle; section 4): every
// E and B value of an x line takes the value one cell further along +x, and the last
// value of the line (x = n for the x-node components Ey, Ez, Bx, x = n - 1/2 for the
// x-half components Ex, By, Bz) becomes zero.  One warp per padded (y, z) line, so the
// y and z ghost lines move with the lines they copy; the line is moved in place 32
// values at a time (each chunk is read before any of it is written, and the next chunk
// starts past what this one wrote).
template <typename T> struct ShiftArgs {
    T* F[6];
    int last[6];   // the last moved x index of each component
};

template <typename T>
__global__ void __launch_bounds__(128) k_window_shift(Geom g, ShiftArgs<T> S) {
    const int lane = threadIdx.x & 31;
    const long long line = blockIdx.x * 4LL + (threadIdx.x >> 5);
    if (line >= (long long)g.Gy * g.Gz) return;   // whole warps
    T* L = S.F[blockIdx.y] + line * g.Px;          // L[i + 1] holds x = i, i = -1 .. Px - 2
    const int last = S.last[blockIdx.y];
    for (int x0 = 0; x0 <= last; x0 += 32) {
        const int i = x0 + lane;
        const T v = i < last ? L[i + 2] : T(0);
        __syncwarp();
        if (i <= last) L[i + 1] = v;
        __syncwarp();
    }
}

template <typename T>
static pic_status window_shift_t(pic_ctx* c) {
    const Geom& g = c->g;
    ShiftArgs<T> S;
    for (int k = 0; k < 3; ++k) {
        S.F[k] = static_cast<T*>(c->E[k]);
        S.F[3 + k] = static_cast<T*>(c->B[k]);
    }
    // x nodes: Ey, Ez (E) and Bx (B); x halves: Ex, By, Bz
    const int n = g.n[0];
    const int last[6] = {n - 1, n, n, n, n - 1, n - 1};
    for (int k = 0; k < 6; ++k) S.last[k] = last[k];
    const long long lines = (long long)g.Gy * g.Gz;
    dim3 grid((unsigned)((lines + 3) / 4), 6);
    LaunchScope ls(c, KC_OTHER);
    k_window_shift<T><<<grid, 128, 0, c->stream>>>(g, S);
    GBPIC_CHECK(c, cudaGetLastError());
    return PIC_OK;
}

pic_status launch_window_shift(pic_ctx* c) {
    return c->prec == PIC_FP64 ? window_shift_t<double>(c) : window_shift_t<float>(c);
}

// ---------------------------------------------------------------------------
// Compensated binomial current filter (section 2.2 "compensated smoothing", section 2.6
// current filtering; the paper gives no scheme): along each dimension one convolution
// of every J component with the kernel K (p binomial stencils (1/4, 1/2, 1/4), then the
// compensator (-p/4, 1 + p/2, -p/4)); periodic dimensions wrap, an open x counts the
// values outside x = 0 .. n - 1 as zero.  One thread per value; the neighbours along x
// are coalesced, those along y and z are whole x lines apart.
template <typename A> struct FilterArgs {
    const A* src[3];
    A* dst[3];
    double K[2 * MAX_FILTER_PASSES + 3];         // the kernel (FP64 path)
    long long Kn[2 * MAX_FILTER_PASSES + 3];     // its numerators over 2^shift (fixed-point path)
    int shift;
    int h;
};

// One filtered value: FP64 sum on the FP64 path; on the FP32 path's 64-bit fixed-point J
// the exact integer sum of the numerators (128-bit), rounded once to the J unit (ties up)
// — the kernel's weights are dyadic, so nothing else is rounded.
// On the fixed-point path each tap splits the 64-bit value into its signed high and
// unsigned low 32-bit halves and adds kn times each into a 64-bit sum (|kn| < 2^21, so
// neither sum can overflow in 2H + 1 <= 19 taps); the halves are joined once, exactly,
// in 128 bits.
struct FixedSum {
    long long hi = 0, lo = 0;
};
struct FilterSum {
    __device__ static __forceinline__ double tap(double acc, double k, long long, double v) { return acc + k * v; }
    __device__ static __forceinline__ FixedSum tap(FixedSum acc, double, long long kn, long long v) {
        const int k32 = (int)kn;
        acc.hi += (long long)(int)(v >> 32) * k32;
        acc.lo += (long long)(unsigned)(v & 0xffffffffLL) * k32;
        return acc;
    }
    __device__ static __forceinline__ double finish(double acc, int) { return acc; }
    __device__ static __forceinline__ long long finish(FixedSum acc, int shift) {
        const __int128 total = ((__int128)acc.hi << 32) + acc.lo;
        return (long long)((total + ((__int128)1 << (shift - 1))) >> shift);
    }
};
template <typename A> struct FilterAcc;
template <> struct FilterAcc<double> { using t = double; };
template <> struct FilterAcc<long long> { using t = FixedSum; };


// Thread (i, j, k) of component c: blockIdx.x covers x in chunks of 128, blockIdx.y is
// y, blockIdx.z is z + n_z c.  Neighbours along `dim` at stride `stride` (values); H is
// the kernel's half width, so the 2H + 1 taps are unrolled and their loads overlap.
template <typename A, int H>
__global__ void __launch_bounds__(128) k_filter_dim(Geom g, FilterArgs<A> F, int dim) {
    const int i = blockIdx.x * 128 + threadIdx.x;
    if (i >= g.n[0]) return;
    const int j = blockIdx.y, comp = blockIdx.z / g.n[2], k = blockIdx.z - comp * g.n[2];
    const int at = dim == 0 ? i : (dim == 1 ? j : k);
    const int nd = dim == 0 ? g.n[0] : (dim == 1 ? g.n[1] : g.n[2]);
    const long long stride = dim == 0 ? 1LL : (dim == 1 ? (long long)g.n[0] : (long long)g.n[0] * g.n[1]);
    const long long e = g.cidx(i, j, k);
    // (selects, not an indexed parameter array, which would be copied to local memory)
    const A* src = comp == 0 ? F.src[0] : (comp == 1 ? F.src[1] : F.src[2]);
    A* dst = comp == 0 ? F.dst[0] : (comp == 1 ? F.dst[1] : F.dst[2]);
    const A* line = src + (e - (long long)at * stride);   // the value at position 0 along dim
    const bool bounded = dim == 0 && g.open_x;
    A v[2 * H + 1];
#pragma unroll
    for (int t = 0; t <= 2 * H; ++t) {
        int q = at + t - H;
        bool in = true;
        if (bounded) {
            in = q >= 0 && q < nd;                  // zero outside an open x
        } else if (nd > H) {
            q += q < 0 ? nd : (q >= nd ? -nd : 0);  // one wrap suffices
        } else {
            q %= nd;
            if (q < 0) q += nd;
        }
        v[t] = in ? line[(long long)q * stride] : A(0);
    }
    typename FilterAcc<A>::t sum{};
#pragma unroll
    for (int t = 0; t <= 2 * H; ++t) sum = FilterSum::tap(sum, F.K[t], F.Kn[t], v[t]);
    dst[e] = FilterSum::finish(sum, F.shift);
}

template <typename A, int H>
static void launch_filter_h(pic_ctx* c, dim3 grid, const FilterArgs<A>& F, int dim) {
    k_filter_dim<A, H><<<grid, 128, 0, c->stream>>>(c->g, F, dim);
}

template <typename A>
static void launch_filter(pic_ctx* c, dim3 grid, const FilterArgs<A>& F, int dim) {
    static_assert(MAX_FILTER_PASSES == 8, "half widths 1 .. 9 below");
    switch (F.h) {
        case 1: launch_filter_h<A, 1>(c, grid, F, dim); break;
        case 2: launch_filter_h<A, 2>(c, grid, F, dim); break;
        case 3: launch_filter_h<A, 3>(c, grid, F, dim); break;
        case 4: launch_filter_h<A, 4>(c, grid, F, dim); break;
        case 5: launch_filter_h<A, 5>(c, grid, F, dim); break;
        case 6: launch_filter_h<A, 6>(c, grid, F, dim); break;
        case 7: launch_filter_h<A, 7>(c, grid, F, dim); break;
        case 8: launch_filter_h<A, 8>(c, grid, F, dim); break;
        default: launch_filter_h<A, 9>(c, grid, F, dim); break;
    }
}

template <typename T>
static pic_status current_filter_t(pic_ctx* c) {
    using A = typename JTraits<T>::acc_t;
    const Geom& g = c->g;
    for (int k = 0; k < 3; ++k) {
        if (!c->Jtmp[k]) {
            c->Jtmp[k] = dev_alloc(c, sizeof(long long) * (size_t)g.N);
            if (!c->Jtmp[k]) return PIC_ERR_OOM;
        }
    }
    FilterArgs<A> F;
    F.shift = 2 * (c->filter_passes + c->filter_compensate);   // the kernel's weights are k / 4^stages
    for (int m = 0; m < 2 * c->filter_h + 1; ++m) {
        F.K[m] = c->filter_K[m];
        F.Kn[m] = (long long)std::llround(std::ldexp(c->filter_K[m], F.shift));   // exact
    }
    F.h = c->filter_h;
    if (g.n[1] > 65535 || 3LL * g.n[2] > 65535) {
        c->err = "current filter: n[1] <= 65535 and n[2] <= 21845";
        return PIC_ERR_ARG;
    }
    const dim3 grid((unsigned)((g.n[0] + 127) / 128), (unsigned)g.n[1], (unsigned)(3 * g.n[2]));
    for (int dim = 0; dim < 3; ++dim) {   // x, y, z; each pass writes the other J set
        for (int k = 0; k < 3; ++k) {
            F.src[k] = static_cast<const A*>(c->J[k]);
            F.dst[k] = static_cast<A*>(c->Jtmp[k]);
        }
        {
            LaunchScope ls(c, KC_OTHER);
            launch_filter<A>(c, grid, F, dim);
            GBPIC_CHECK(c, cudaGetLastError());
        }
        for (int k = 0; k < 3; ++k) std::swap(c->J[k], c->Jtmp[k]);
    }
    return PIC_OK;
}

pic_status launch_current_filter(pic_ctx* c) {
    return c->prec == PIC_FP64 ? current_filter_t<double>(c) : current_filter_t<float>(c);
}

// ---------------------------------------------------------------------------
// Perfectly conducting wall planes and the waveguide port (section 3.2 verification:
// the TE10 mode of a conducting rectangular guide driven at its input plane).  After
// Ampere's law (and the Mur faces): the port sets Ez(0, j, k) = amp sin(m pi j / n_y)
// and Ey(0, j, k) = 0 on the face x = 0 (amp = e0 g(t) sin(omega t), from the host);
// then the wall planes hold their tangential E at zero: Ex, Ez on y = 0, Ex, Ey on
// z = 0.  In the periodic y (z) the plane y = 0 is both walls of a guide of width n_y.
// Every value is stored with its y and z ghost images; the wall kernel also covers the
// x ghost columns (they hold copies of the same, zero, values).
template <typename T>
__global__ void k_port(Geom g, T* Ey, T* Ez, double amp, int mode_y) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (j >= g.n[1]) return;
    const double prof = sin(mode_y * 3.14159265358979323846 * (double)j / g.n[1]);
    store1_yz(g, Ey, 0, j, k, T(0));
    store1_yz(g, Ez, 0, j, k, (T)(amp * prof));
}

template <typename T>
__global__ void k_pec(Geom g, T* Ex, T* Ey, T* Ez, int pec_y, int pec_z) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x - 1;   // padded x: -1 .. Px - 2
    if (i > g.Px - 2) return;
    const int t = blockIdx.y;
    if (pec_y && t < g.n[2]) {
        store1_yz(g, Ex, i, 0, t, T(0));
        store1_yz(g, Ez, i, 0, t, T(0));
    }
    if (pec_z && t < g.n[1]) {
        store1_yz(g, Ex, i, t, 0, T(0));
        store1_yz(g, Ey, i, t, 0, T(0));
    }
}

template <typename T>
static pic_status guide_t(pic_ctx* c) {
    const Geom& g = c->g;
    if (c->port_on) {
        const pic_port_desc& P = c->port;
        const double t = (c->step + 1) * c->desc.dt;   // the time of the new E
        const double amp = P.e0 * (1.0 - std::exp(-t / P.tau)) * std::sin(P.omega * t);
        LaunchScope ls(c, KC_OTHER);
        k_port<T><<<dim3((g.n[1] + 127) / 128, g.n[2]), 128, 0, c->stream>>>(g, (T*)c->E[1], (T*)c->E[2], amp,
                                                                              P.mode_y);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    if (c->pec_y || c->pec_z) {
        LaunchScope ls(c, KC_OTHER);
        k_pec<T><<<dim3((g.Px + 127) / 128, std::max(g.n[1], g.n[2])), 128, 0, c->stream>>>(
            g, (T*)c->E[0], (T*)c->E[1], (T*)c->E[2], c->pec_y, c->pec_z);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    return PIC_OK;
}

pic_status launch_guide(pic_ctx* c) {
    return c->prec == PIC_FP64 ? guide_t<double>(c) : guide_t<float>(c);
}

pic_status launch_open_x_before_ampere(pic_ctx* c) {
    return c->prec == PIC_FP64 ? open_before_t<double>(c) : open_before_t<float>(c);
}
pic_status launch_open_x_after_ampere(pic_ctx* c) {
    return c->prec == PIC_FP64 ? open_after_t<double>(c) : open_after_t<float>(c);
}

}  // namespace gbpic

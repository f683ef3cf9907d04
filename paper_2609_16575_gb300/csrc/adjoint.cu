// Hand-written discrete adjoint of the PIC cycle (KEMPIC-3D section 2.2, Fig. 2) for
// gradients of the final field energy L = U_E + U_B (time level N, B^N of Eq. (21))
// with respect to the initial momenta u^{-1/2} and an initial-field amplitude.
//
// State s^n = (E^n, B^{n-1/2}, X^n, u^{n-1/2}).  One forward cycle is
//   B_n = B^{n-1/2} - h C_E E^n        (h = dt/2; C_E the curl from E to B locations)
//   particles: gather E^n, B_n at X^n; Boris; X^{n+1} = X^n + (dt/d) u/gamma; zigzag J
//   B^{n+1/2} = B_n - h C_E E^n
//   E^{n+1} = E^n + dt (C_B B^{n+1/2} - J)
// On the Yee grid C_B = C_E^T, so the transposed field updates reuse the two curl
// stencils.  With lambdas of s^{n+1} the adjoint step is
//   lB  <- lB + dt C_E lE'            (lambda of B^{n+1/2} = lambda of B_n, field part)
//   lE  <- lE' - h C_B lB             (field part of lambda of E^n)
//   particles, lambda_J = -dt lE': deposit^T (derivatives of the zigzag fluxes and
//     weights), position update^T, Boris^T, gather^T (scatter into lE, lB and the
//     derivative of the interpolation weights)
//   lE  <- lE - h C_B lB              (from B_n = B^{n-1/2} - h C_E E^n)
// The host loop keeps a full-state snapshot every K steps, recomputes each segment
// forward, and runs the adjoint steps in reverse.  The field adjoints, the gather^T
// accumulators and the parameter-gradient reductions are FP64; the per-particle
// Jacobian products and the particles' adjoint state use the working precision.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pic_internal.cuh"

namespace gbpic {

struct SpeciesSnap {
    void* part = nullptr;
    void* counts = nullptr;
    void* ctr = nullptr;
    void* spill = nullptr;
    int cur = 0;
};

struct Snapshot {
    void* fields[6] = {};
    std::vector<SpeciesSnap> sp;
    int64_t step = 0;
};

// The backward host loop's device buffers.
struct AdjBuffers {
    double* lE[3] = {};
    double* lB[3] = {};
    void* lJ[3] = {};       // -dt lambda_E^{n+1} in the working precision
    double* accE[3] = {};   // accE[0..2] and accB[0..2] are one contiguous block
    double* accB[3] = {};
    void* Bn[3] = {};
    std::vector<void*> lX, lU;   // the particles' adjoint state, working precision
    std::vector<double*> conv;   // FP64 copies of lU for dL_du (FP32 path only)
    double* stage = nullptr;     // the directions E_dir, B_dir and the dL_dA sum
};

struct AdjointState {
    int N = 0, K = 1;
    double loss = 0;
    std::vector<Snapshot> ckpt;
    std::vector<Snapshot> seg;
    Snapshot final_;
    AdjBuffers buf;
    void* block = nullptr;                 // the one device allocation all of the above use
    std::vector<int64_t> species_loaded;   // n_loaded per species at the forward pass
    bool ready = false;
};

static size_t field_bytes(pic_ctx* c) { return (size_t)c->g.padded_size() * c->esize; }
static int ntiles(pic_ctx* c) { return c->g.nt[0] * c->g.nt[1] * c->g.nt[2]; }
static size_t rec_bytes(pic_ctx* c) { return c->prec == PIC_FP64 ? sizeof(Rec<double>) : sizeof(Rec<float>); }

// Several device-to-device copies in one launch (a snapshot is a dozen buffers; at the
// sizes of the differentiable run one launch per buffer cost more than the bytes).
// Blocks stride over each item in the widest units that both its addresses allow:
// 16-byte vectors when both are 16-byte aligned, then 4-byte words when both are
// 4-byte aligned, then bytes (a snapshot's tile counts sit at 4-byte offsets).
constexpr int MCOPY_MAX = 16;
struct CopyList {
    const void* src[MCOPY_MAX];
    void* dst[MCOPY_MAX];
    long long bytes[MCOPY_MAX];
    int n;
};
__global__ void k_multi_copy(CopyList L) {
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
    for (int it = 0; it < L.n; ++it) {
        const uintptr_t al = reinterpret_cast<uintptr_t>(L.src[it]) | reinterpret_cast<uintptr_t>(L.dst[it]);
        const long long nb = L.bytes[it];
        long long done = 0;
        if ((al & 15) == 0) {
            const uint4* s = static_cast<const uint4*>(L.src[it]);
            uint4* d = static_cast<uint4*>(L.dst[it]);
            const long long n16 = nb >> 4;
            for (long long e = t0; e < n16; e += st) d[e] = s[e];
            done = n16 << 4;
        }
        if ((al & 3) == 0) {
            const unsigned* s = static_cast<const unsigned*>(L.src[it]);
            unsigned* d = static_cast<unsigned*>(L.dst[it]);
            const long long nw = nb >> 2;
            for (long long e = (done >> 2) + t0; e < nw; e += st) d[e] = s[e];
            done = nw << 2;
        }
        const unsigned char* s = static_cast<const unsigned char*>(L.src[it]);
        unsigned char* d = static_cast<unsigned char*>(L.dst[it]);
        for (long long e = done + t0; e < nb; e += st) d[e] = s[e];
    }
}
struct MultiCopy {
    pic_ctx* c;
    CopyList L{};
    pic_status st = PIC_OK;
    explicit MultiCopy(pic_ctx* cc) : c(cc) {}
    void add(void* dst, const void* src, size_t bytes) {
        if (st != PIC_OK || bytes == 0) return;
        if (L.n == MCOPY_MAX) flush();
        L.src[L.n] = src;
        L.dst[L.n] = dst;
        L.bytes[L.n] = (long long)bytes;
        ++L.n;
    }
    pic_status flush() {
        if (st == PIC_OK && L.n > 0) {
            LaunchScope ls(c, KC_OTHER);
            k_multi_copy<<<1024, 256, 0, c->stream>>>(L);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) st = cuda_fail(c, e, "k_multi_copy");
        }
        L.n = 0;
        return st;
    }
};

// The adjoint's device memory is one block, reserved by pic_adjoint_forward and carved
// into the checkpoints, the segment's recomputed states, the final state and the
// backward pass's buffers: cudaMalloc and cudaFree synchronise the device and take tens
// of microseconds each, and a backward pass had made some two hundred of them.  Carve
// runs twice: once with a null base to size the block, once to hand out its pieces
// (each 256-byte aligned).
struct Carve {
    unsigned char* base = nullptr;
    size_t off = 0;
    void* take(size_t n) {
        void* r = base ? base + off : nullptr;
        off += (n + 255) & ~size_t(255);
        return r;
    }
};

static void snap_carve(pic_ctx* c, Carve& cv, Snapshot& S) {
    for (int k = 0; k < 6; ++k) S.fields[k] = cv.take(field_bytes(c));
    S.sp.resize(c->species.size());
    for (size_t i = 0; i < c->species.size(); ++i) {
        SpeciesDev& s = c->species[i];
        SpeciesSnap& z = S.sp[i];
        z.part = cv.take(s.pbytes);
        z.counts = cv.take((2 + TILE_CELLS) * sizeof(int) * ntiles(c));
        z.ctr = cv.take(sizeof(Counters));
        z.spill = cv.take(rec_bytes(c) * s.spill_cap);
    }
}

static void buffers_carve(pic_ctx* c, Carve& cv, AdjBuffers& b) {
    const size_t pb = sizeof(double) * (size_t)c->g.padded_size();
    const size_t cb = sizeof(double) * (size_t)c->g.N;
    const size_t fb = field_bytes(c);
    double* acc6 = static_cast<double*>(cv.take(6 * cb));   // accE[0..2], accB[0..2], contiguous
    for (int k = 0; k < 3; ++k) {
        b.lE[k] = static_cast<double*>(cv.take(pb));
        b.lB[k] = static_cast<double*>(cv.take(pb));
        b.accE[k] = acc6 ? acc6 + k * (size_t)c->g.N : nullptr;
        b.accB[k] = acc6 ? acc6 + (3 + k) * (size_t)c->g.N : nullptr;
        b.Bn[k] = cv.take(fb);
        b.lJ[k] = cv.take(fb);
    }
    b.lX.clear();
    b.lU.clear();
    b.conv.clear();
    for (auto& s : c->species) {
        const size_t m = 3 * (size_t)std::max<int64_t>(s.n_loaded, 1);
        b.lX.push_back(cv.take(c->esize * m));
        b.lU.push_back(cv.take(c->esize * m));
        b.conv.push_back(c->esize == sizeof(double) ? nullptr : static_cast<double*>(cv.take(sizeof(double) * m)));
    }
    b.stage = static_cast<double*>(cv.take(sizeof(double) * (6 * (size_t)c->g.N + 1)));
}

// Sizes and reserves the block for the state's checkpoints and segment states.
static pic_status adjoint_reserve(pic_ctx* c, AdjointState& S) {
    size_t total = 0;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            S.block = dev_alloc(c, total);
            if (!S.block) return PIC_ERR_OOM;
        }
        Carve cv;
        cv.base = static_cast<unsigned char*>(S.block);
        for (auto& z : S.ckpt) snap_carve(c, cv, z);
        for (auto& z : S.seg) snap_carve(c, cv, z);
        snap_carve(c, cv, S.final_);
        buffers_carve(c, cv, S.buf);
        total = cv.off;
    }
    S.species_loaded.clear();
    for (auto& s : c->species) S.species_loaded.push_back(s.n_loaded);
    return PIC_OK;
}

static pic_status snap_save(pic_ctx* c, Snapshot& S) {
    const size_t fb = field_bytes(c);
    MultiCopy M(c);
    for (int k = 0; k < 3; ++k) {
        M.add(S.fields[k], c->E[k], fb);
        M.add(S.fields[3 + k], c->B[k], fb);
    }
    for (size_t i = 0; i < c->species.size(); ++i) {
        SpeciesDev& s = c->species[i];
        SpeciesSnap& z = S.sp[i];
        z.cur = s.cur;
        M.add(z.part, s.base[s.cur], s.pbytes);
        M.add(z.counts, s.count, sizeof(int) * ntiles(c));
        M.add(static_cast<int*>(z.counts) + ntiles(c), s.holes, sizeof(int) * ntiles(c));
        M.add(static_cast<int*>(z.counts) + 2 * ntiles(c), s.hist[s.cur], sizeof(int) * TILE_CELLS * ntiles(c));
        M.add(z.ctr, s.ctr, sizeof(Counters));
        M.add(z.spill, s.spill, rec_bytes(c) * s.spill_cap);
    }
    const pic_status st = M.flush();
    if (st != PIC_OK) return st;
    S.step = c->step;
    return PIC_OK;
}

static pic_status snap_restore(pic_ctx* c, const Snapshot& S) {
    const size_t fb = field_bytes(c);
    MultiCopy M(c);
    for (int k = 0; k < 3; ++k) {
        M.add(c->E[k], S.fields[k], fb);
        M.add(c->B[k], S.fields[3 + k], fb);
    }
    for (size_t i = 0; i < c->species.size(); ++i) {
        SpeciesDev& s = c->species[i];
        const SpeciesSnap& z = S.sp[i];
        s.cur = z.cur;
        M.add(s.base[s.cur], z.part, s.pbytes);
        M.add(s.count, z.counts, sizeof(int) * ntiles(c));
        M.add(s.holes, static_cast<const int*>(z.counts) + ntiles(c), sizeof(int) * ntiles(c));
        M.add(s.hist[s.cur], static_cast<const int*>(z.counts) + 2 * ntiles(c), sizeof(int) * TILE_CELLS * ntiles(c));
        M.add(s.ctr, z.ctr, sizeof(Counters));
        M.add(s.spill, z.spill, rec_bytes(c) * s.spill_cap);
    }
    pic_status st = M.flush();
    if (st != PIC_OK) return st;
    for (int k = 0; k < 3; ++k) GBPIC_CHECK(c, cudaMemsetAsync(c->J[k], 0, sizeof(long long) * (size_t)c->g.N, c->stream));
    c->step = S.step;
    c->j_dirty = false;
    return PIC_OK;
}

// ---------------------------------------------------------------------------
// Adjoint kernels: per-particle arithmetic in the working precision, FP64 adjoint state
// and accumulation.

template <typename T> struct AdjArgs {
    Geom g;
    ParticleArrays<T> pa;
    const Rec<T>* spill;
    const Counters* ctr;   // the spill count of the state: ctr->spill_count[parity]
    int parity;
    int spill_cap;
    const T* E[3];      // E^n
    const T* Bn[3];     // B_n = B^{n-1/2} - dt/2 curl E^n
    const T* lJ[3];     // lambda_J = -dt lambda of E^{n+1} (padded), in the working precision
    double* accE[3];    // gather^T accumulators (compact)
    double* accB[3];
    T* lX;              // 3 x nload lambda of positions (cell units), load order
    T* lU;              // 3 x nload lambda of momenta
    long long nload;
    double eps, dt, dtd[3], C[3];   // C = q / (dt d_p d_r)
};

// Value and gradient (w.r.t. the three fractional coordinates) of a trilinear
// interpolation of F from base (b0, b1, b2) with fractions s, in arithmetic C.
template <typename T, typename C>
__device__ __forceinline__ C interp_grad(const Geom& g, const T* F, const int b[3], const C s[3], C grad[3]) {
    C f[2][2][2];
    // the eight samples from the base's padded index (local -1 .. n: no wrap needed)
    const long long base = g.pidx(b[0], b[1], b[2]), sy = g.Px, sz = (long long)g.Px * g.Gy;
    #pragma unroll
    for (int cc = 0; cc < 2; ++cc)
        #pragma unroll
        for (int bb = 0; bb < 2; ++bb)
            #pragma unroll
            for (int aa = 0; aa < 2; ++aa) f[cc][bb][aa] = (C)F[base + aa + bb * sy + cc * sz];
    const C w0[2] = {C(1) - s[0], s[0]}, w1[2] = {C(1) - s[1], s[1]}, w2[2] = {C(1) - s[2], s[2]};
    C v = 0, g0 = 0, g1 = 0, g2 = 0;
    #pragma unroll
    for (int cc = 0; cc < 2; ++cc)
        #pragma unroll
        for (int bb = 0; bb < 2; ++bb)
            #pragma unroll
            for (int aa = 0; aa < 2; ++aa) {
                const C x = f[cc][bb][aa];
                v += w0[aa] * w1[bb] * w2[cc] * x;
                g0 += (aa ? C(1) : C(-1)) * w1[bb] * w2[cc] * x;
                g1 += w0[aa] * (bb ? C(1) : C(-1)) * w2[cc] * x;
                g2 += w0[aa] * w1[bb] * (cc ? C(1) : C(-1)) * x;
            }
    grad[0] = g0;
    grad[1] = g1;
    grad[2] = g2;
    return v;
}

// lam times the trilinear weights of component comp, through Add(comp, x, y, z, value)
// at the eight nodes from base b (the value in arithmetic C; the accumulator decides
// its own precision).
template <typename C, typename AddFn>
__device__ __forceinline__ void scatter_trilinear(AddFn Add, int comp, const int b[3], const C s[3], C lam) {
    if (lam == C(0)) return;
    const C w0[2] = {C(1) - s[0], s[0]}, w1[2] = {C(1) - s[1], s[1]}, w2[2] = {C(1) - s[2], s[2]};
    #pragma unroll
    for (int cc = 0; cc < 2; ++cc)
        #pragma unroll
        for (int bb = 0; bb < 2; ++bb)
            #pragma unroll
            for (int aa = 0; aa < 2; ++aa) Add(comp, b[0] + aa, b[1] + bb, b[2] + cc, lam * w0[aa] * w1[bb] * w2[cc]);
}

// Derivatives of S = sum_q L_q v_q(F, W) for one straight segment (the 12 edge
// values of segment_values) with respect to its fluxes F and midpoint offsets W.
template <typename C>
__device__ __forceinline__ void segment_vjp(const C Cw[3], const C F[3], const C W[3], const C L[12], C gF[3], C gW[3]) {
    const C wx1 = W[0], wy1 = W[1], wz1 = W[2], wx0 = 1 - wx1, wy0 = 1 - wy1, wz0 = 1 - wz1;
    const C Ax = L[0] * wy0 * wz0 + L[1] * wy1 * wz0 + L[2] * wy0 * wz1 + L[3] * wy1 * wz1;
    const C Ay = L[4] * wx0 * wz0 + L[5] * wx1 * wz0 + L[6] * wx0 * wz1 + L[7] * wx1 * wz1;
    const C Az = L[8] * wx0 * wy0 + L[9] * wx1 * wy0 + L[10] * wx0 * wy1 + L[11] * wx1 * wy1;
    const C Gx = L[0] - L[1] - L[2] + L[3];
    const C Gy = L[4] - L[5] - L[6] + L[7];
    const C Gz = L[8] - L[9] - L[10] + L[11];
    const C Fx = F[0], Fy = F[1], Fz = F[2];
    const C Cx = Cw[0], Cy = Cw[1], Cz = Cw[2];
    const C t = C(1) / C(12);
    gF[0] = Cx * (Ax + Fy * Fz * Gx * t) + Cy * Fy * Fz * Gy * t + Cz * Fz * Fy * Gz * t;
    gF[1] = Cy * (Ay + Fx * Fz * Gy * t) + Cx * Fx * Fz * Gx * t + Cz * Fz * Fx * Gz * t;
    gF[2] = Cz * (Az + Fx * Fy * Gz * t) + Cx * Fx * Fy * Gx * t + Cy * Fy * Fx * Gy * t;
    gW[0] = Cy * Fy * ((L[5] - L[4]) * wz0 + (L[7] - L[6]) * wz1) + Cz * Fz * ((L[9] - L[8]) * wy0 + (L[11] - L[10]) * wy1);
    gW[1] = Cx * Fx * ((L[1] - L[0]) * wz0 + (L[3] - L[2]) * wz1) + Cz * Fz * ((L[10] - L[8]) * wx0 + (L[11] - L[9]) * wx1);
    gW[2] = Cx * Fx * ((L[2] - L[0]) * wy0 + (L[3] - L[1]) * wy1) + Cy * Fy * ((L[6] - L[4]) * wx0 + (L[7] - L[5]) * wx1);
}

template <typename C>
__device__ __forceinline__ void cross3(const C a[3], const C b[3], C o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// The particle part of one adjoint step.  The per-particle Jacobian products and the
// particles' adjoint state carried across steps (lambda of positions and momenta, like
// the forward particle state) run in the working precision C (FP32 on the FP32 path,
// where FP64 arithmetic would run on the GPU's narrow FP64 pipe); the field
// accumulators and the parameter gradients are FP64 on both paths.
// The trilinear stencil of field component comp (E_c half a cell along c, B_c half a
// cell along the other two) at a particle in cell gc with in-cell offsets d1: the base
// node b and the fractions s (section 2.5's staggered CIC weights).
template <typename C>
__device__ __forceinline__ void adj_stencil(const int gc[3], const C d1[3], int comp, int b[3], C s[3]) {
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
        const bool half = comp < 3 ? k == comp : k != comp - 3;
        if (!half) {
            b[k] = gc[k];
            s[k] = d1[k];
        } else if (d1[k] >= C(0.5)) {
            b[k] = gc[k];
            s[k] = d1[k] - C(0.5);
        } else {
            b[k] = gc[k] - 1;
            s[k] = d1[k] + C(0.5);
        }
    }
}

// Returns in lam the adjoint of the six gathered components (lambda_E, lambda_B at the
// particle), which the caller scatters through the stencils of adj_stencil (gather^T),
// and updates the particle's own adjoint state in lX, lU.
template <typename T, typename C>
__device__ void adjoint_particle(const AdjArgs<T>& A, int gx, int gy, int gz, const C d1[3], const C u0[3], C w, int id,
                                 C lam[6]) {
    const Geom& g = A.g;
    const int gc[3] = {gx, gy, gz};
    // ---- forward recompute: staggered gather with weights and their gradients
    C val[6], grad[6][3];
    #pragma unroll
    for (int comp = 0; comp < 6; ++comp) {
        int cb[3];
        C cs[3];
        adj_stencil(gc, d1, comp, cb, cs);
        const T* F = comp < 3 ? A.E[comp] : A.Bn[comp - 3];
        val[comp] = interp_grad<T, C>(g, F, cb, cs, grad[comp]);
    }
    const C Ep[3] = {val[0], val[1], val[2]}, Bp[3] = {val[3], val[4], val[5]};
    // Boris with its intermediates (section 2.4)
    const C eps = (C)A.eps;
    C um[3], t[3], s[3], up[3], upl[3], un[3], tmp[3];
    #pragma unroll
    for (int k = 0; k < 3; ++k) um[k] = u0[k] + eps * Ep[k];
    const C gm = sqrt(C(1) + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    #pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = eps * Bp[k] / gm;
    const C t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    const C f = C(2) / (C(1) + t2);
    #pragma unroll
    for (int k = 0; k < 3; ++k) s[k] = f * t[k];
    cross3(um, t, tmp);
    #pragma unroll
    for (int k = 0; k < 3; ++k) up[k] = um[k] + tmp[k];
    cross3(up, s, tmp);
    #pragma unroll
    for (int k = 0; k < 3; ++k) upl[k] = um[k] + tmp[k];
    #pragma unroll
    for (int k = 0; k < 3; ++k) un[k] = upl[k] + eps * Ep[k];
    const C gn = sqrt(C(1) + un[0] * un[0] + un[1] * un[1] + un[2] * un[2]);
    const C ig = C(1) / gn;
    // move and zigzag relay (cell-relative, as the forward kernels)
    C d2[3], F1[3], F2[3], W1[3], W2[3];
    int st[3];
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
        st[k] = advance(d1[k], (C)A.dtd[k] * un[k] * ig, d2[k]);
        st[k] = st[k] > 1 ? 1 : (st[k] < -1 ? -1 : st[k]);
        relay(d1[k], d2[k], st[k], F1[k], F2[k], W1[k], W2[k]);
    }
    // ---- deposit^T: lambda_J = -dt lambda_E^{n+1} at the edges of both segment cells
    // the edges of the start cell and of the (wrapped) end cell: padded indices from each
    // cell's origin (edges up to local n, inside the padded range with its valid ghosts)
    C L1[12], L2[12];
    {
        const long long sy = g.Px, sz = (long long)g.Px * g.Gy;
        const long long o1 = g.pidx(gx, gy, gz);
        const long long o2 = g.pidx(wrap1(gx + st[0], g.n[0]), wrap1(gy + st[1], g.n[1]), wrap1(gz + st[2], g.n[2]));
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            int comp, ex, ey, ez;
            slot_edge(q, 0, 0, 0, comp, ex, ey, ez);
            const long long off = ex + ey * sy + ez * sz;
            L1[q] = (C)A.lJ[comp][o1 + off];
            L2[q] = (C)A.lJ[comp][o2 + off];
        }
    }
    const C Cw[3] = {(C)A.C[0] * w, (C)A.C[1] * w, (C)A.C[2] * w};
    C gF1[3], gW1[3], gF2[3], gW2[3];
    segment_vjp(Cw, F1, W1, L1, gF1, gW1);
    segment_vjp(Cw, F2, W2, L2, gF2, gW2);
    C lx1c[3], lx2c[3];
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (st[k] == 0) {   // F1 = F2 = (x2 - x1)/2, W1 = (3 x1 + x2)/4, W2 = (x1 + 3 x2)/4
            lx1c[k] = C(-0.5) * (gF1[k] + gF2[k]) + C(0.75) * gW1[k] + C(0.25) * gW2[k];
            lx2c[k] = C(0.5) * (gF1[k] + gF2[k]) + C(0.25) * gW1[k] + C(0.75) * gW2[k];
        } else {            // F1 = +-(1 - x1) ..., W1 = (x1 [+1])/2; F2 = x2 [-1], W2 = (x2 [+1])/2
            lx1c[k] = -gF1[k] + C(0.5) * gW1[k];
            lx2c[k] = gF2[k] + C(0.5) * gW2[k];
        }
    }
    // ---- the adjoint of the next state (FP64), and the position update
    // X^{n+1} = X^n + dtd u / gamma
    C lx1[3], lun[3], a[3];
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
        const C lx2 = lx2c[k] + (C)A.lX[k * A.nload + id];
        lx1[k] = lx1c[k] + lx2;
        a[k] = lx2 * (C)A.dtd[k];
    }
    const C adot = a[0] * un[0] + a[1] * un[1] + a[2] * un[2];
    #pragma unroll
    for (int k = 0; k < 3; ++k) lun[k] = (C)A.lU[k * A.nload + id] + (a[k] - un[k] * adot * ig * ig) * ig;
    // ---- Boris^T
    C lum[3], lup[3], ls[3], lt[3], lE[3], lB[3];
    #pragma unroll
    for (int k = 0; k < 3; ++k) lum[k] = lun[k];           // upl = um + up x s, lambda_upl = lun
    cross3(s, lun, lup);                                     // lambda_up = s x lambda_upl
    cross3(lun, up, ls);                                     // lambda_s = lambda_upl x up
    cross3(t, lup, tmp);                                     // up = um + um x t
    #pragma unroll
    for (int k = 0; k < 3; ++k) lum[k] += lup[k] + tmp[k];
    cross3(lup, um, lt);
    const C lst = ls[0] * t[0] + ls[1] * t[1] + ls[2] * t[2];   // s = f t, f = 2 / (1 + t.t)
    #pragma unroll
    for (int k = 0; k < 3; ++k) lt[k] += f * ls[k] - f * f * lst * t[k];
    #pragma unroll
    for (int k = 0; k < 3; ++k) lB[k] = eps / gm * lt[k];    // t = eps B / gm
    const C lgm = -(lt[0] * t[0] + lt[1] * t[1] + lt[2] * t[2]) / gm;
    #pragma unroll
    for (int k = 0; k < 3; ++k) lum[k] += lgm * um[k] / gm;   // gm = sqrt(1 + um.um)
    #pragma unroll
    for (int k = 0; k < 3; ++k) lE[k] = eps * (lun[k] + lum[k]);   // um = u + eps E and the final kick
    // ---- gather^T
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
        C acc = 0;
        #pragma unroll
        for (int c = 0; c < 3; ++c) acc += lE[c] * grad[c][k] + lB[c] * grad[3 + c][k];
        lx1[k] += acc;
    }
    #pragma unroll
    for (int c = 0; c < 3; ++c) {
        lam[c] = lE[c];
        lam[3 + c] = lB[c];
    }
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
        A.lX[k * A.nload + id] = (T)lx1[k];
        A.lU[k * A.nload + id] = (T)lum[k];
    }
}

// gather^T of one particle through Add(comp, x, y, z, value).
template <typename C, typename AddFn>
__device__ __forceinline__ void scatter_particle(AddFn Add, const int gc[3], const C d1[3], const C lam[6]) {
    #pragma unroll
    for (int comp = 0; comp < 6; ++comp) {
        int b[3];
        C sf[3];
        adj_stencil(gc, d1, comp, b, sf);
        scatter_trilinear(Add, comp, b, sf, lam[comp]);
    }
}

// Each CTA takes a chunk of adj_chunk<T>() slots of one tile (blocks beyond the tiles'
// chunks take the spill list).  The gather^T contributions of the chunk are summed in a
// shared box of the tile's nodes -1..8 per dimension and added to the global FP64
// accumulators once per node.  The box holds the working precision: FP64 sums on the
// FP64 path, FP32 sums of at most one chunk's terms on the FP32 path (whose per-particle
// Jacobians are FP32 already), where FP64 additions would run on the GPU's narrow FP64
// pipe.  Lane l of warp w handles slots (chunk / 32) l + w + 8 m: the lanes of a warp sit
// one or two cells apart in the cell-sorted segment, so they rarely add to the same node
// at once (shared floating-point additions to one address serialise).  The FP64 kernel
// holds one CTA per SM (its registers), so its chunks are half as long: twice the CTAs
// leave a shorter tail.  (64-bit fixed-point sums in two 32-bit words with native
// shared reductions, as the tile kernel's current tile, ran no faster on the FP32 path:
// the fixed-point unit needs the chunk's largest lambda before the first addition, so
// every particle's lambdas had to be staged in shared memory first.)
constexpr int AB = 10;   // nodes per dimension of the shared adjoint box
constexpr int ADJ_NB = 6 * AB * AB * AB;
template <typename T> __host__ __device__ constexpr int adj_chunk() { return sizeof(T) == sizeof(double) ? 512 : 1024; }
template <typename T>
__global__ void __launch_bounds__(256) k_adj_particles(AdjArgs<T> A, int chunks_per_tile) {
    constexpr int CH = adj_chunk<T>();
    __shared__ T sacc[ADJ_NB];
    const Geom& g = A.g;
    const int nt = g.nt[0] * g.nt[1] * g.nt[2];
    auto gadd = [&](int comp, int x, int y, int z, T v) {
        double* acc = comp < 3 ? A.accE[comp] : A.accB[comp - 3];
        atomicAdd(acc + g.cidx(wrap_idx(x, g.n[0]), wrap_idx(y, g.n[1]), wrap_idx(z, g.n[2])), (double)v);
    };
    const long long nblk_tiles = (long long)nt * chunks_per_tile;
    if (blockIdx.x >= nblk_tiles) {   // the spill list
        const int nsp = min(A.ctr->spill_count[A.parity], A.spill_cap);
        for (long long i = (blockIdx.x - nblk_tiles) * blockDim.x + threadIdx.x; i < nsp;
             i += (gridDim.x - nblk_tiles) * blockDim.x) {
            const Rec<T> r = A.spill[i];
            const int gc[3] = {r.cell % g.n[0], (r.cell / g.n[0]) % g.n[1], r.cell / (g.n[0] * g.n[1])};
            T lam[6];
            adjoint_particle<T, T>(A, gc[0], gc[1], gc[2], r.d, r.u, r.w, r.id, lam);
            scatter_particle(gadd, gc, r.d, lam);
        }
        return;
    }
    const int t = blockIdx.x / chunks_per_tile, chunk = blockIdx.x % chunks_per_tile;
    const int cnt = min(A.pa.count[t], A.pa.cap[t]);
    const int i0 = chunk * CH;
    if (i0 >= cnt) return;
    const int tx = t % g.nt[0], ty = (t / g.nt[0]) % g.nt[1], tz = t / (g.nt[0] * g.nt[1]);
    const int ox = tx * TILE, oy = ty * TILE, oz = tz * TILE;
    for (int i = threadIdx.x; i < ADJ_NB; i += blockDim.x) sacc[i] = T(0);
    __syncthreads();
    auto sadd = [&](int comp, int x, int y, int z, T v) {
        atomicAdd(sacc + ((comp * AB + (z - oz + 1)) * AB + (y - oy + 1)) * AB + (x - ox + 1), v);
    };
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int m = 0; m < CH / 256; ++m) {
        const int i = i0 + (CH / 32) * lane + warp + 8 * m;
        if (i >= cnt) continue;
        const long long p = (long long)A.pa.seg_start[t] + i;
        const int lc = A.pa.cell[p];
        if (lc < 0) continue;
        const int gc[3] = {ox + (lc & 7), oy + ((lc >> 3) & 7), oz + (lc >> 6)};
        const T d1[3] = {A.pa.d[0][p], A.pa.d[1][p], A.pa.d[2][p]};
        const T u0[3] = {A.pa.u[0][p], A.pa.u[1][p], A.pa.u[2][p]};
        T lam[6];
        adjoint_particle<T, T>(A, gc[0], gc[1], gc[2], d1, u0, A.pa.w[p], A.pa.id[p], lam);
        scatter_particle(sadd, gc, d1, lam);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ADJ_NB; e += blockDim.x) {
        const T v = sacc[e];
        if (v == T(0)) continue;
        const int lx = e % AB, ly = (e / AB) % AB, lz = (e / (AB * AB)) % AB, comp = e / (AB * AB * AB);
        gadd(comp, ox + lx - 1, oy + ly - 1, oz + lz - 1, v);
    }
}

// dst_k (working precision, padded) = scale * src_k (FP64, padded), ghosts included.
template <typename T>
__global__ void k_to_working3(long long n, const double* s0, const double* s1, const double* s2, T* d0, T* d1, T* d2,
                              double scale) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        d0[e] = (T)(scale * s0[e]);
        d1[e] = (T)(scale * s1[e]);
        d2[e] = (T)(scale * s2[e]);
    }
}

// dst (FP64, padded) = scale * src (working precision, padded), ghosts included.
template <typename T>
__global__ void k_scale_copy(long long n, const T* src, double* dst, double scale) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        dst[e] = scale * (double)src[e];
}


// lE += accE and lB += accB (acc: the six compact accumulators in one block), ghost
// images included.
__global__ void k_merge6(Geom g, double* e0, double* e1, double* e2, double* b0, double* b1, double* b2,
                         const double* acc) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.N; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % g.n[0]), j = (int)((e / g.n[0]) % g.n[1]), k = (int)(e / ((long long)g.n[0] * g.n[1]));
        const long long p = g.pidx(i, j, k);
        store3(g, e0, e1, e2, i, j, k, e0[p] + acc[e], e1[p] + acc[g.N + e], e2[p] + acc[2 * g.N + e]);
        store3(g, b0, b1, b2, i, j, k, b0[p] + acc[3 * g.N + e], b1[p] + acc[4 * g.N + e], b2[p] + acc[5 * g.N + e]);
    }
}

// sum over cells of lE . Ed + lB . Bd (Ed, Bd compact, FP64)
__global__ void k_dot(Geom g, const double* lE0, const double* lE1, const double* lE2, const double* lB0,
                      const double* lB1, const double* lB2, const double* Ed, const double* Bd, double* out) {
    double acc = 0;
    const long long N = g.N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % g.n[0]), j = (int)((e / g.n[0]) % g.n[1]), k = (int)(e / ((long long)g.n[0] * g.n[1]));
        const long long p = g.pidx(i, j, k);
        if (Ed) acc += lE0[p] * Ed[e] + lE1[p] * Ed[N + e] + lE2[p] * Ed[2 * N + e];
        if (Bd) acc += lB0[p] * Bd[e] + lB1[p] * Bd[N + e] + lB2[p] * Bd[2 * N + e];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(out, acc);
}

// ---------------------------------------------------------------------------
// The backward host loop.

// The particle arrays of a snapshot: the live block layout the snapshot copied, rebased
// onto the snapshot's copy, with its tile counts and holes.
template <typename T>
static ParticleArrays<T> snap_view(pic_ctx* c, SpeciesDev& s, const SpeciesSnap& z) {
    ParticleArrays<T> v = z.cur == s.cur ? arrays<T>(s) : arrays_alt<T>(s);
    const unsigned char* b0 = static_cast<const unsigned char*>(s.base[z.cur]);
    unsigned char* nb = static_cast<unsigned char*>(z.part);
    auto rebase = [&](auto* p) {
        return reinterpret_cast<decltype(p)>(nb + (reinterpret_cast<const unsigned char*>(p) - b0));
    };
    v.cell = rebase(v.cell);
    for (int k = 0; k < 3; ++k) {
        v.d[k] = rebase(v.d[k]);
        v.u[k] = rebase(v.u[k]);
    }
    v.w = rebase(v.w);
    v.id = rebase(v.id);
    v.count = static_cast<int*>(z.counts);
    v.holes = static_cast<int*>(z.counts) + ntiles(c);
    return v;
}

// One adjoint step at the state held by snapshot Z (read in place: the live state is
// not touched).
template <typename T>
static pic_status adjoint_step_t(pic_ctx* c, AdjBuffers& b, const Snapshot& Z) {
    const double dt = c->desc.dt, h = 0.5 * dt;
    {   // lambda_J = -dt lambda_E^{n+1} (lE before this step's field updates), once per
        // node in the working precision
        LaunchScope ls(c, KC_OTHER);
        k_to_working3<T><<<1024, 256, 0, c->stream>>>(c->g.padded_size(), b.lE[0], b.lE[1], b.lE[2],
                                                      static_cast<T*>(b.lJ[0]), static_cast<T*>(b.lJ[1]),
                                                      static_cast<T*>(b.lJ[2]), -dt);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    // lB += dt C_E lE  (the Faraday stencil computes B - coef curl E)
    pic_status st = curl_to_b<double>(c, b.lE, b.lB, -dt);
    if (st != PIC_OK) return st;
    // lE -= h C_B lB
    st = curl_to_e<double>(c, b.lE, b.lB, -h);
    if (st != PIC_OK) return st;
    // B_n of this state
    const size_t fb = (size_t)c->g.padded_size() * sizeof(T);
    T* Bn[3];
    T* E[3];
    {
        MultiCopy M(c);
        for (int k = 0; k < 3; ++k) {
            Bn[k] = static_cast<T*>(b.Bn[k]);
            E[k] = static_cast<T*>(Z.fields[k]);
            M.add(Bn[k], Z.fields[3 + k], fb);
        }
        st = M.flush();
        if (st != PIC_OK) return st;
    }
    st = curl_to_b<T>(c, E, Bn, h);
    if (st != PIC_OK) return st;
    // the six gather^T accumulators are one block
    GBPIC_CHECK(c, cudaMemsetAsync(b.accE[0], 0, 6 * sizeof(double) * (size_t)c->g.N, c->stream));
    for (size_t si = 0; si < c->species.size(); ++si) {
        SpeciesDev& s = c->species[si];
        const SpeciesSnap& z = Z.sp[si];
        AdjArgs<T> A{};
        A.g = c->g;
        A.pa = snap_view<T>(c, s, z);
        A.spill = static_cast<const Rec<T>*>(z.spill);
        A.ctr = static_cast<const Counters*>(z.ctr);
        A.parity = (int)(Z.step & 1);
        A.spill_cap = s.spill_cap;
        for (int k = 0; k < 3; ++k) {
            A.E[k] = E[k];
            A.Bn[k] = Bn[k];
            A.lJ[k] = static_cast<const T*>(b.lJ[k]);
            A.accE[k] = b.accE[k];
            A.accB[k] = b.accB[k];
        }
        A.lX = static_cast<T*>(b.lX[si]);
        A.lU = static_cast<T*>(b.lU[si]);
        A.nload = s.n_loaded;
        A.eps = s.q * dt / (2.0 * s.m);
        A.dt = dt;
        const double* d = c->desc.d;
        for (int k = 0; k < 3; ++k) A.dtd[k] = dt / d[k];
        A.C[0] = s.q / (dt * d[1] * d[2]);
        A.C[1] = s.q / (dt * d[2] * d[0]);
        A.C[2] = s.q / (dt * d[0] * d[1]);
        int maxcap = 0;
        for (int cap : s.h_cap) maxcap = std::max(maxcap, cap);
        const int chunks = std::max(1, (maxcap + adj_chunk<T>() - 1) / adj_chunk<T>());
        // the spill list's blocks (its count stays on the device: no host round trip)
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->desc.device);
        // (the list is usually empty or short: a few blocks stride over it)
        const int spill_blocks = std::max(1, std::min((s.spill_cap + 255) / 256, std::max(sms / 4, 1)));
        const long long blocks = (long long)ntiles(c) * chunks + spill_blocks;
        LaunchScope ls(c, KC_OTHER);
        k_adj_particles<T><<<(unsigned)blocks, 256, 0, c->stream>>>(A, chunks);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    {
        LaunchScope ls(c, KC_OTHER);
        k_merge6<<<1024, 256, 0, c->stream>>>(c->g, b.lE[0], b.lE[1], b.lE[2], b.lB[0], b.lB[1], b.lB[2], b.accE[0]);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    // lE -= h C_B lB  (B_n = B^{n-1/2} - h C_E E^n)
    return curl_to_e<double>(c, b.lE, b.lB, -h);
}

static void adjoint_release(pic_ctx* c) {
    AdjointState* S = static_cast<AdjointState*>(c->adj);
    if (!S) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    dev_free(c, S->block);
    delete S;
    c->adj = nullptr;
}

template <typename T>
static pic_status backward_t(pic_ctx* c, AdjointState& S, const double* Ed, const double* Bd, double* dL_dA,
                             double* const* dL_du, int devptr) {
    AdjBuffers& b = S.buf;
    const size_t cb = sizeof(double) * (size_t)c->g.N;
    const size_t fb = (size_t)c->g.padded_size() * sizeof(T);
    for (size_t si = 0; si < c->species.size(); ++si) {
        const size_t nb = sizeof(T) * 3 * std::max<int64_t>(c->species[si].n_loaded, 1);
        GBPIC_CHECK(c, cudaMemsetAsync(b.lX[si], 0, nb, c->stream));
        GBPIC_CHECK(c, cudaMemsetAsync(b.lU[si], 0, nb, c->stream));
    }
    // the final state and the adjoint of L = 1/2 dV sum (E^N^2 + B_N^2)
    pic_status st = snap_restore(c, S.final_);
    if (st != PIC_OK) return st;
    const double dV = c->desc.d[0] * c->desc.d[1] * c->desc.d[2], h = 0.5 * c->desc.dt;
    T* E[3];
    T* Bn[3];
    for (int k = 0; k < 3; ++k) {
        E[k] = static_cast<T*>(c->E[k]);
        Bn[k] = static_cast<T*>(b.Bn[k]);
        GBPIC_CHECK(c, cudaMemcpyAsync(Bn[k], c->B[k], fb, cudaMemcpyDeviceToDevice, c->stream));
    }
    st = curl_to_b<T>(c, E, Bn, h);
    if (st != PIC_OK) return st;
    {
        LaunchScope ls(c, KC_OTHER);
        for (int k = 0; k < 3; ++k) {
            k_scale_copy<T><<<1024, 256, 0, c->stream>>>(c->g.padded_size(), Bn[k], b.lB[k], dV);
            k_scale_copy<T><<<1024, 256, 0, c->stream>>>(c->g.padded_size(), E[k], b.lE[k], dV);
        }
        GBPIC_CHECK(c, cudaGetLastError());
    }
    st = curl_to_e<double>(c, b.lE, b.lB, -h);
    if (st != PIC_OK) return st;
    // segments in reverse: restore, recompute the states, adjoint steps backwards.  A
    // segment's recomputation and adjoint steps (some 16 launches per step) run as one
    // captured CUDA graph when the capture succeeds (the host side of the segment runs
    // while capturing; the graph of one segment is captured while the previous one runs)
    const int nseg = (int)S.ckpt.size();
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int a = sg * S.K, e = std::min(S.N, a + S.K);
        st = snap_restore(c, S.ckpt[sg]);
        if (st != PIC_OK) return st;
        auto segment = [&]() -> pic_status {
            for (int n = a; n < e; ++n) {
                pic_status r = snap_save(c, S.seg[n - a]);
                if (r != PIC_OK) return r;
                if (n < e - 1) {
                    r = step_once(c, nullptr, false);
                    if (r != PIC_OK) return r;
                }
            }
            for (int n = e - 1; n >= a; --n) {
                const pic_status r = adjoint_step_t<T>(c, b, S.seg[n - a]);
                if (r != PIC_OK) return r;
            }
            return PIC_OK;
        };
        const int64_t step0 = c->step, launches0 = c->launches;
        std::vector<int> cur0;
        for (auto& sp : c->species) cur0.push_back(sp.cur);
        bool done = false;
        st = run_as_graph(c, segment, &done);
        if (st != PIC_OK) return st;
        if (!done) {   // the capture failed: the host state back, the segment launched directly
            c->step = step0;
            c->launches = launches0;
            for (size_t i = 0; i < c->species.size(); ++i) c->species[i].cur = cur0[i];
            st = segment();
            if (st != PIC_OK) return st;
        }
    }
    // parameter gradients (FP64)
    if (dL_dA) {
        double* stage = b.stage;
        const double* dEd = Ed;
        const double* dBd = Bd;
        if (!devptr) {
            if (Ed) GBPIC_CHECK(c, cudaMemcpyAsync(stage, Ed, 3 * cb, cudaMemcpyHostToDevice, c->stream));
            if (Bd) GBPIC_CHECK(c, cudaMemcpyAsync(stage + 3 * c->g.N, Bd, 3 * cb, cudaMemcpyHostToDevice, c->stream));
            dEd = Ed ? stage : nullptr;
            dBd = Bd ? stage + 3 * c->g.N : nullptr;
        }
        double* out = stage + 6 * c->g.N;
        GBPIC_CHECK(c, cudaMemsetAsync(out, 0, sizeof(double), c->stream));
        {
            LaunchScope ls(c, KC_OTHER);
            k_dot<<<1024, 256, 0, c->stream>>>(c->g, b.lE[0], b.lE[1], b.lE[2], b.lB[0], b.lB[1], b.lB[2], dEd, dBd, out);
            GBPIC_CHECK(c, cudaGetLastError());
        }
        GBPIC_CHECK(c, cudaMemcpyAsync(dL_dA, out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    if (dL_du) {
        for (size_t si = 0; si < c->species.size(); ++si) {
            if (!dL_du[si]) continue;
            // the momenta's adjoint in FP64 (a converted copy on the FP32 path)
            const long long m = 3 * c->species[si].n_loaded;
            const double* src = static_cast<const double*>(b.lU[si]);
            if (sizeof(T) != sizeof(double) && m > 0) {
                double* conv = b.conv[si];
                LaunchScope ls(c, KC_OTHER);
                k_scale_copy<T><<<1024, 256, 0, c->stream>>>(m, static_cast<const T*>(b.lU[si]), conv, 1.0);
                GBPIC_CHECK(c, cudaGetLastError());
                src = conv;
            }
            GBPIC_CHECK(c, cudaMemcpyAsync(dL_du[si], src, sizeof(double) * m,
                                           devptr ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
        }
    }
    // leave the context at the final state
    st = snap_restore(c, S.final_);
    if (st != PIC_OK) return st;
    GBPIC_CHECK(c, cudaStreamSynchronize(c->stream));
    return PIC_OK;
}

}  // namespace gbpic

using namespace gbpic;

extern "C" {

pic_status pic_adjoint_forward(pic_ctx* c, int32_t nsteps, int32_t ckpt_every, double* loss) {
    if (!c || nsteps < 1 || ckpt_every < 1 || !loss) return PIC_ERR_ARG;
    if (!c->desc.track_ids || c->species.empty() || c->g.open_x || c->filter_passes > 0 ||
        c->deposit != PIC_DEPOSIT_ZIGZAG || c->shape != PIC_SHAPE_CIC) {
        c->err = "pic_adjoint_forward needs track_ids, at least one species, a periodic box, no current filter "
                 "and the ZigZag deposit with the CIC shape";
        return PIC_ERR_STATE;
    }
    DeviceScope dscope_(c->desc.device);
    adjoint_release(c);
    AdjointState* S = new AdjointState();
    c->adj = S;
    S->N = nsteps;
    S->K = ckpt_every;
    S->ckpt.resize((nsteps + ckpt_every - 1) / ckpt_every);
    S->seg.resize(std::min(nsteps, ckpt_every));
    pic_status st0 = adjoint_reserve(c, *S);
    if (st0 != PIC_OK) return st0;
    update_jscale(c);
    if (c->j_dirty) {
        for (int k = 0; k < 3; ++k)
            GBPIC_CHECK(c, cudaMemsetAsync(c->J[k], 0, sizeof(long long) * (size_t)c->g.N, c->stream));
        c->j_dirty = false;
    }
    for (int n = 0; n < nsteps; ++n) {
        pic_status st;
        if (n % ckpt_every == 0) {
            st = snap_save(c, S->ckpt[n / ckpt_every]);
            if (st != PIC_OK) return st;
        }
        st = step_once(c, nullptr, false);
        if (st != PIC_OK) return st;
    }
    pic_status st = snap_save(c, S->final_);
    if (st != PIC_OK) return st;
    double UE = 0, UB = 0;
    st = energy_sums(c, &UE, &UB);
    if (st != PIC_OK) return st;
    st = pic_sync(c);
    if (st != PIC_OK) return st;
    S->loss = UE + UB;
    S->ready = true;
    *loss = S->loss;
    return PIC_OK;
}

pic_status pic_adjoint_backward(pic_ctx* c, const double* E_dir, const double* B_dir, double* dL_dA,
                                double* const* dL_du, int32_t device_pointers) {
    if (!c) return PIC_ERR_ARG;
    AdjointState* S = static_cast<AdjointState*>(c->adj);
    if (!S || !S->ready) {
        c->err = "pic_adjoint_backward needs a preceding pic_adjoint_forward";
        return PIC_ERR_STATE;
    }
    bool same = S->species_loaded.size() == c->species.size();
    for (size_t i = 0; same && i < c->species.size(); ++i) same = S->species_loaded[i] == c->species[i].n_loaded;
    if (!same) {
        c->err = "pic_adjoint_backward: the species changed since pic_adjoint_forward";
        return PIC_ERR_STATE;
    }
    DeviceScope dscope_(c->desc.device);
    pic_status st = c->prec == PIC_FP64 ? backward_t<double>(c, *S, E_dir, B_dir, dL_dA, dL_du, device_pointers)
                                        : backward_t<float>(c, *S, E_dir, B_dir, dL_dA, dL_du, device_pointers);
    if (st != PIC_OK) return st;
    return pic_sync(c);
}

pic_status pic_adjoint_run(pic_ctx* c, int32_t nsteps, int32_t ckpt_every, const double* E_dir, const double* B_dir,
                           double* loss, double* dL_dA, double* const* dL_du, int32_t device_pointers) {
    pic_status st = pic_adjoint_forward(c, nsteps, ckpt_every, loss);
    if (st != PIC_OK) return st;
    return pic_adjoint_backward(c, E_dir, B_dir, dL_dA, dL_du, device_pointers);
}

}  // extern "C"

namespace gbpic {
void adjoint_free(pic_ctx* c) { adjoint_release(c); }
}  // namespace gbpic

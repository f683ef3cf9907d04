// Set-up and read-out kernels: species loading (positions to cell + offset in the
// working precision, counting sort into 8^3-cell tile segments ordered by cell),
// field upload with ghost images, and FP64 read-out of fields and particles.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "pic_internal.cuh"

namespace gbpic {


// Position (cell units) -> global cell and in-cell offset in the working precision.
// An offset that rounds to 1 moves to offset 0 of the next cell.  Returns false for
// a position outside [0, n) or not finite.
template <typename T>
__device__ __forceinline__ bool locate(const Geom& g, const double X[3], int c[3], T dl[3]) {
    for (int k = 0; k < 3; ++k) {
        const double x = X[k];
        if (!(x >= 0.0 && x < (double)g.n[k])) return false;
        double f = floor(x);
        int ci = (int)f;
        T o = (T)(x - f);
        if (o >= T(1)) {
            o = T(0);
            ci += 1;
            if (ci >= g.n[k]) ci = 0;
        }
        c[k] = ci;
        dl[k] = o;
    }
    return true;
}

__device__ __forceinline__ int key_of(const Geom& g, const int c[3]) {
    const int t = ((c[2] >> 3) * g.nt[1] + (c[1] >> 3)) * g.nt[0] + (c[0] >> 3);
    return t * TILE_CELLS + ((c[0] & 7) | ((c[1] & 7) << 3) | ((c[2] & 7) << 6));
}

template <typename T>
__global__ void k_keys(Geom g, const double* X, const double* w, long long n, int* hist, int* bad,
                       unsigned long long* wmax_bits) {
    // the largest weight: a thread's own maximum, then the warp's, then one atomic per
    // warp (positive doubles order like their bit patterns)
    unsigned long long wbits = 0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const double Xp[3] = {X[p], X[n + p], X[2 * n + p]};
        int c[3];
        T dl[3];
        const double wp = w[p];
        if (!locate<T>(g, Xp, c, dl) || !(wp > 0.0) || !isfinite(wp)) {
            atomicOr(bad, 1);
            continue;
        }
        atomicAdd(hist + key_of(g, c), 1);
        const unsigned long long b = (unsigned long long)__double_as_longlong(wp);
        wbits = b > wbits ? b : wbits;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, wbits, o);
        wbits = v > wbits ? v : wbits;
    }
    if ((threadIdx.x & 31) == 0 && wbits) atomicMax(wmax_bits, wbits);
}

template <typename T>
__global__ void k_scatter(Geom g, const double* X, const double* U, const double* w, const double* ids, long long n,
                          int* keypos, ParticleArrays<T> pa, int track_ids) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const double Xp[3] = {X[p], X[n + p], X[2 * n + p]};
        int c[3];
        T dl[3];
        if (!locate<T>(g, Xp, c, dl)) continue;
        const int key = key_of(g, c);
        const int q = atomicAdd(keypos + key, 1);
        pa.cell[q] = key & (TILE_CELLS - 1);
        for (int k = 0; k < 3; ++k) {
            pa.d[k][q] = dl[k];
            pa.u[k][q] = (T)U[k * n + p];
        }
        pa.w[q] = (T)w[p];
        if (track_ids) pa.id[q] = ids ? (int)ids[p] : (int)p;
    }
}

// Loader staging record: one particle's working-precision state in one aligned
// 32-byte (FP32) or 64-byte (FP64) block, so that the scatter into random slots writes
// whole DRAM sectors (eight separate 4-byte stores per particle leave eight partly
// written sectors); k_unpack then writes the SoA arrays tile by tile, coalesced.
template <typename T> struct LoadRec;
template <> struct alignas(32) LoadRec<float> {
    int cell;
    float d[3], u[3], w;
};
template <> struct alignas(64) LoadRec<double> {
    int cell, id;
    double d[3], u[3], w;
};
static_assert(sizeof(LoadRec<float>) == 32 && sizeof(LoadRec<double>) == 64, "loader records fill whole sectors");

template <typename T>
__global__ void k_scatter_rec(Geom g, const double* X, const double* U, const double* w, const double* ids, long long n,
                              int* keypos, LoadRec<T>* recs, int* id_out, int track_ids) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const double Xp[3] = {X[p], X[n + p], X[2 * n + p]};
        int c[3];
        T dl[3];
        if (!locate<T>(g, Xp, c, dl)) continue;
        const int key = key_of(g, c);
        const int q = atomicAdd(keypos + key, 1);
        LoadRec<T> r;
        r.cell = key & (TILE_CELLS - 1);
        for (int k = 0; k < 3; ++k) {
            r.d[k] = dl[k];
            r.u[k] = (T)U[k * n + p];
        }
        r.w = (T)w[p];
        const int id = ids ? (int)ids[p] : (int)p;
        if constexpr (sizeof(T) == 8) r.id = id;
        else if (track_ids) id_out[q] = id;
        recs[q] = r;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_unpack_rec(const LoadRec<T>* recs, ParticleArrays<T> pa, int ntile, int track_ids) {
    for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int cnt = pa.count[t];
        const long long s0 = pa.seg_start[t];
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const long long q = s0 + i;
            const LoadRec<T> r = recs[q];
            pa.cell[q] = r.cell;
            for (int k = 0; k < 3; ++k) {
                pa.d[k][q] = r.d[k];
                pa.u[k][q] = r.u[k];
            }
            pa.w[q] = r.w;
            if constexpr (sizeof(T) == 8) {
                if (track_ids) pa.id[q] = r.id;
            }
        }
    }
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// ids: optional FP64 load-order ids of the particles (host or device like X), for a
// restored state; without them particle p gets id p.
template <typename T>
static pic_status load_t(pic_ctx* c, const pic_species_desc* d, SpeciesDev& s, const double* ids_in) {
    const long long n = d->n;
    const Geom& g = c->g;
    const int ntile = g.nt[0] * g.nt[1] * g.nt[2];
    const long long nkeys = (long long)ntile * TILE_CELLS;
    // staging: device copies of the FP64 inputs
    const double *X = d->X, *U = d->u, *W = d->w, *IDS = ids_in;
    double* stage = nullptr;
    if (!d->device_pointers && n > 0) {
        stage = static_cast<double*>(dev_alloc(c, sizeof(double) * (ids_in ? 8 : 7) * n));
        if (!stage) return PIC_ERR_OOM;
        GBPIC_CHECK(c, cudaMemcpyAsync(stage, d->X, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream));
        GBPIC_CHECK(c, cudaMemcpyAsync(stage + 3 * n, d->u, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream));
        GBPIC_CHECK(c, cudaMemcpyAsync(stage + 6 * n, d->w, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
        if (ids_in)
            GBPIC_CHECK(c, cudaMemcpyAsync(stage + 7 * n, ids_in, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
        X = stage;
        U = stage + 3 * n;
        W = stage + 6 * n;
        IDS = ids_in ? stage + 7 * n : nullptr;
    }
    int* hist = static_cast<int*>(dev_alloc(c, sizeof(int) * (nkeys + 2) + 8));
    if (!hist) return PIC_ERR_OOM;
    int* bad = hist + nkeys;
    unsigned long long* wmax_bits = reinterpret_cast<unsigned long long*>(hist + nkeys + 2);
    GBPIC_CHECK(c, cudaMemsetAsync(hist, 0, sizeof(int) * (nkeys + 2) + 8, c->stream));
    const int grid = 1024;
    if (n > 0) {
        LaunchScope ls(c, KC_OTHER);
        k_keys<T><<<grid, 256, 0, c->stream>>>(g, X, W, n, hist, bad, wmax_bits);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    std::vector<int> h_hist(nkeys);
    int h_bad = 0;
    unsigned long long h_wbits = 0;
    GBPIC_CHECK(c, cudaMemcpyAsync(h_hist.data(), hist, sizeof(int) * nkeys, cudaMemcpyDeviceToHost, c->stream));
    GBPIC_CHECK(c, cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GBPIC_CHECK(c, cudaMemcpyAsync(&h_wbits, wmax_bits, 8, cudaMemcpyDeviceToHost, c->stream));
    GBPIC_CHECK(c, cudaStreamSynchronize(c->stream));
    if (h_bad) {
        c->err = "pic_load_species: a position is outside [0, n) or a weight is not positive and finite";
        dev_free(c, hist);
        if (stage) dev_free(c, stage);
        return PIC_ERR_ARG;
    }
    double wmax = 0;
    memcpy(&wmax, &h_wbits, 8);
    // tile capacities and segment starts (host), key positions within segments; the
    // species that a moving window fills gets room for the plateau density in every
    // tile (the plasma comes in at the window's front)
    const double slack = d->capacity_slack > 0 ? d->capacity_slack : 0.25;
    const bool window_species = c->window_on && c->window.species == (int)c->species.size() - 1;
    const long long window_ppc =
        window_species ? (long long)c->window.ppc[0] * c->window.ppc[1] * c->window.ppc[2] : 0;
    s.h_seg_start.assign(ntile, 0);
    s.h_cap.assign(ntile, 0);
    std::vector<int> h_count(ntile, 0);
    long long total = 0;
    for (int t = 0; t < ntile; ++t) {
        long long cnt = 0;
        for (int l = 0; l < TILE_CELLS; ++l) cnt += h_hist[(size_t)t * TILE_CELLS + l];
        long long want = cnt;
        if (window_species) {
            const int tx = t % g.nt[0], ty = (t / g.nt[0]) % g.nt[1], tz = t / (g.nt[0] * g.nt[1]);
            const long long cells = (long long)std::min(TILE, g.n[0] - tx * TILE) *
                                    std::min(TILE, g.n[1] - ty * TILE) * std::min(TILE, g.n[2] - tz * TILE);
            want = std::max(want, cells * window_ppc);
        }
        long long cap = want + std::max<long long>((long long)std::ceil(slack * want), 32);
        cap = (cap + 31) / 32 * 32;
        s.h_seg_start[t] = (int)total;
        s.h_cap[t] = (int)cap;
        h_count[t] = (int)cnt;
        total += cap;
        if (total > 0x7fffff00LL) {
            c->err = "pic_load_species: more than 2^31 particle slots";
            return PIC_ERR_ARG;
        }
    }
    std::vector<int> h_keypos(nkeys);
    for (int t = 0; t < ntile; ++t) {
        int acc = s.h_seg_start[t];
        for (int l = 0; l < TILE_CELLS; ++l) {
            h_keypos[(size_t)t * TILE_CELLS + l] = acc;
            acc += h_hist[(size_t)t * TILE_CELLS + l];
        }
    }
    GBPIC_CHECK(c, cudaMemcpyAsync(hist, h_keypos.data(), sizeof(int) * nkeys, cudaMemcpyHostToDevice, c->stream));
    // two particle blocks (current and sort target), each: cell, d[3], u[3], w, id;
    // then the per-tile segment arrays and the counters, shared by both blocks
    const size_t cap = (size_t)total;
    const size_t a_int = align256(cap * sizeof(int)), a_t = align256(cap * sizeof(T));
    const size_t pbytes = a_int * 2 + a_t * 7;
    const size_t bytes = pbytes + align256(sizeof(int) * ntile) * 4 + align256(sizeof(Counters));
    unsigned char* base = static_cast<unsigned char*>(dev_alloc(c, bytes));
    unsigned char* base2 = static_cast<unsigned char*>(dev_alloc(c, pbytes));
    s.hist[0] = static_cast<int*>(dev_alloc(c, sizeof(int) * (size_t)nkeys));
    s.hist[1] = static_cast<int*>(dev_alloc(c, sizeof(int) * (size_t)nkeys));
    if (!base || !base2 || !s.hist[0] || !s.hist[1]) return PIC_ERR_OOM;
    s.base[0] = base;
    s.base[1] = base2;
    s.pbytes = pbytes;
    s.cur = 0;
    size_t off = pbytes;
    s.seg_start = reinterpret_cast<int*>(base + off); off += align256(sizeof(int) * ntile);
    s.count = reinterpret_cast<int*>(base + off); off += align256(sizeof(int) * ntile);
    s.cap = reinterpret_cast<int*>(base + off); off += align256(sizeof(int) * ntile);
    s.holes = reinterpret_cast<int*>(base + off); off += align256(sizeof(int) * ntile);
    s.ctr = reinterpret_cast<Counters*>(base + off);
    for (int b = 0; b < 2; ++b) {
        ParticleArrays<T>& pb = b == 0 ? arrays<T>(s) : arrays_alt<T>(s);
        unsigned char* blk = static_cast<unsigned char*>(s.base[b]);
        size_t o = 0;
        pb.cell = reinterpret_cast<int*>(blk + o); o += a_int;
        for (int k = 0; k < 3; ++k) { pb.d[k] = reinterpret_cast<T*>(blk + o); o += a_t; }
        for (int k = 0; k < 3; ++k) { pb.u[k] = reinterpret_cast<T*>(blk + o); o += a_t; }
        pb.w = reinterpret_cast<T*>(blk + o); o += a_t;
        pb.id = reinterpret_cast<int*>(blk + o); o += a_int;
        pb.seg_start = s.seg_start;
        pb.count = s.count;
        pb.cap = s.cap;
        pb.holes = s.holes;
    }
    ParticleArrays<T>& pa = arrays<T>(s);
    GBPIC_CHECK(c, cudaMemsetAsync(base, 0, bytes, c->stream));
    GBPIC_CHECK(c, cudaMemcpyAsync(s.seg_start, s.h_seg_start.data(), sizeof(int) * ntile, cudaMemcpyHostToDevice, c->stream));
    GBPIC_CHECK(c, cudaMemcpyAsync(s.count, h_count.data(), sizeof(int) * ntile, cudaMemcpyHostToDevice, c->stream));
    GBPIC_CHECK(c, cudaMemcpyAsync(s.cap, s.h_cap.data(), sizeof(int) * ntile, cudaMemcpyHostToDevice, c->stream));
    // the cell histogram of the loaded block (the tile kernel's output ranges)
    GBPIC_CHECK(c, cudaMemcpyAsync(s.hist[0], h_hist.data(), sizeof(int) * nkeys, cudaMemcpyHostToDevice, c->stream));
    if (n > 0) {
        // through whole-sector staging records when their buffer can be had, else
        // straight into the SoA arrays
        LoadRec<T>* recs = static_cast<LoadRec<T>*>(dev_alloc(c, sizeof(LoadRec<T>) * (size_t)total));
        LaunchScope ls(c, KC_OTHER);
        if (recs) {
            k_scatter_rec<T><<<grid, 256, 0, c->stream>>>(g, X, U, W, IDS, n, hist, recs, pa.id, c->desc.track_ids);
            GBPIC_CHECK(c, cudaGetLastError());
            k_unpack_rec<T><<<std::min(ntile, 65535), 256, 0, c->stream>>>(recs, pa, ntile, c->desc.track_ids);
            GBPIC_CHECK(c, cudaGetLastError());
            GBPIC_CHECK(c, cudaStreamSynchronize(c->stream));
            dev_free(c, recs);
        } else {
            k_scatter<T><<<grid, 256, 0, c->stream>>>(g, X, U, W, IDS, n, hist, pa, c->desc.track_ids);
            GBPIC_CHECK(c, cudaGetLastError());
        }
    }
    // mover and spill lists (a window move sends the first cell column of every tile to
    // the tile before it: an eighth of the particles, plus the new column's plasma)
    s.mover_cap = (int)std::min<long long>(
        d->mover_capacity > 0 ? d->mover_capacity : std::max<long long>(window_species ? total / 4 : n / 4, 65536),
        0x7fffff00LL);
    s.spill_cap = (int)std::min<long long>(d->spill_capacity > 0 ? d->spill_capacity : std::max<long long>(n / 16, 65536),
                                           0x7fffff00LL);
    s.movers = dev_alloc(c, sizeof(Rec<T>) * (size_t)s.mover_cap);
    s.spill = dev_alloc(c, sizeof(Rec<T>) * (size_t)s.spill_cap);
    if (!s.movers || !s.spill) return PIC_ERR_OOM;
    GBPIC_CHECK(c, cudaStreamSynchronize(c->stream));
    dev_free(c, hist);
    if (stage) dev_free(c, stage);
    s.q = d->q;
    s.m = d->m;
    s.n_loaded = n;
    s.cap_total = (int64_t)total;
    // fixed-point unit of J: a bound on one deposit term |q| w / (dt d_p d_r) (x 1.25
    // for the straight-segment correction) maps to 2^JBITS units
    const double* dd = c->desc.d;
    const double dmin2 = std::min(dd[0] * dd[1], std::min(dd[1] * dd[2], dd[2] * dd[0]));
    if (window_species) {   // the heaviest particle the window will bring in
        const pic_window_desc& W = c->window;
        wmax = std::max(wmax, W.density * dd[0] * dd[1] * dd[2] / (double)window_ppc);
    }
    const double bound = std::fabs(d->q) * wmax / (c->desc.dt * dmin2) * 1.25;
    s.jscale = bound > 0 ? bound / std::ldexp(1.0, Prec<T>::JBITS) : 0.0;
    return PIC_OK;
}

pic_status load_species_impl(pic_ctx* c, const pic_species_desc* d, SpeciesDev& s) {
    return c->prec == PIC_FP64 ? load_t<double>(c, d, s, nullptr) : load_t<float>(c, d, s, nullptr);
}

pic_status load_species_ids(pic_ctx* c, const pic_species_desc* d, SpeciesDev& s, const double* ids) {
    return c->prec == PIC_FP64 ? load_t<double>(c, d, s, ids) : load_t<float>(c, d, s, ids);
}

// ---------------------------------------------------------------------------
// Read-out of particles as FP64 rows X, Y, Z, ux, uy, uz, w.

// One CTA of 256 threads per tile; without ids the particles keep their slot order
// (holes skipped by a block-wide prefix count).
template <typename T>
__global__ void __launch_bounds__(256) k_read_tiles(Geom g, ParticleArrays<T> pa, const long long* out_off, double* out,
                                                    long long nout, int use_ids) {
    __shared__ int wtot[8];
    const int ntile = g.nt[0] * g.nt[1] * g.nt[2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int cnt = min(pa.count[t], pa.cap[t]);
        const int tx = t % g.nt[0], ty = (t / g.nt[0]) % g.nt[1], tz = t / (g.nt[0] * g.nt[1]);
        long long written = 0;
        for (int base = 0; base < cnt; base += 256) {
            const int i = base + threadIdx.x;
            const long long p = (long long)pa.seg_start[t] + i;
            const int lc = i < cnt ? pa.cell[p] : HOLE;
            const unsigned bal = __ballot_sync(0xffffffffu, lc >= 0);
            __syncthreads();   // the previous chunk's totals are consumed
            if (lane == 0) wtot[warp] = __popc(bal);
            __syncthreads();
            int before = 0, total = 0;
            for (int w = 0; w < 8; ++w) {
                before += w < warp ? wtot[w] : 0;
                total += wtot[w];
            }
            const long long rank = written + before + __popc(bal & ((1u << lane) - 1u));
            written += total;
            if (lc < 0) continue;
            const long long o = use_ids ? (long long)pa.id[p] : out_off[t] + rank;
            if (o < 0 || o >= nout) continue;
            out[o] = (double)(tx * TILE + (lc & 7)) + (double)pa.d[0][p];
            out[nout + o] = (double)(ty * TILE + ((lc >> 3) & 7)) + (double)pa.d[1][p];
            out[2 * nout + o] = (double)(tz * TILE + (lc >> 6)) + (double)pa.d[2][p];
            out[3 * nout + o] = (double)pa.u[0][p];
            out[4 * nout + o] = (double)pa.u[1][p];
            out[5 * nout + o] = (double)pa.u[2][p];
            out[6 * nout + o] = (double)pa.w[p];
        }
    }
}

template <typename T>
__global__ void k_read_spill(Geom g, const Rec<T>* spill, int nsp, long long base, double* out, long long nout,
                             int use_ids) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsp; i += gridDim.x * blockDim.x) {
        const Rec<T> r = spill[i];
        const long long o = use_ids ? (long long)r.id : base + i;
        if (o < 0 || o >= nout) continue;
        const int gx = r.cell % g.n[0], gy = (r.cell / g.n[0]) % g.n[1], gz = r.cell / (g.n[0] * g.n[1]);
        out[o] = gx + (double)r.d[0];
        out[nout + o] = gy + (double)r.d[1];
        out[2 * nout + o] = gz + (double)r.d[2];
        out[3 * nout + o] = (double)r.u[0];
        out[4 * nout + o] = (double)r.u[1];
        out[5 * nout + o] = (double)r.u[2];
        out[6 * nout + o] = (double)r.w;
    }
}

template <typename T>
static pic_status read_t(pic_ctx* c, SpeciesDev& s, double* out, int64_t nout) {
    const Geom& g = c->g;
    const int ntile = g.nt[0] * g.nt[1] * g.nt[2];
    std::vector<int> h_count(ntile), h_holes(ntile);
    Counters h_ctr;
    GBPIC_CHECK(c, cudaMemcpyAsync(h_count.data(), s.count, sizeof(int) * ntile, cudaMemcpyDeviceToHost, c->stream));
    GBPIC_CHECK(c, cudaMemcpyAsync(h_holes.data(), s.holes, sizeof(int) * ntile, cudaMemcpyDeviceToHost, c->stream));
    GBPIC_CHECK(c, cudaMemcpyAsync(&h_ctr, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream));
    GBPIC_CHECK(c, cudaStreamSynchronize(c->stream));
    std::vector<long long> off(ntile);
    long long acc = 0;
    for (int t = 0; t < ntile; ++t) {
        off[t] = acc;
        acc += std::min(h_count[t], s.h_cap[t]) - h_holes[t];
    }
    long long* d_off = static_cast<long long*>(dev_alloc(c, sizeof(long long) * ntile));
    if (!d_off) return PIC_ERR_OOM;
    GBPIC_CHECK(c, cudaMemcpyAsync(d_off, off.data(), sizeof(long long) * ntile, cudaMemcpyHostToDevice, c->stream));
    const int use_ids = c->desc.track_ids ? 1 : 0;
    {
        LaunchScope ls(c, KC_OTHER);
        k_read_tiles<T><<<1024, 256, 0, c->stream>>>(g, arrays<T>(s), d_off, out, nout, use_ids);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    const int nsp = std::min(h_ctr.spill_count[c->step & 1], s.spill_cap);
    if (nsp > 0) {
        LaunchScope ls(c, KC_OTHER);
        k_read_spill<T><<<256, 256, 0, c->stream>>>(g, static_cast<const Rec<T>*>(s.spill), nsp, acc, out, nout, use_ids);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    GBPIC_CHECK(c, cudaStreamSynchronize(c->stream));
    dev_free(c, d_off);
    return PIC_OK;
}

pic_status get_particles_impl(pic_ctx* c, SpeciesDev& s, double* out_dev, int64_t n_out) {
    return c->prec == PIC_FP64 ? read_t<double>(c, s, out_dev, n_out) : read_t<float>(c, s, out_dev, n_out);
}

int64_t count_alive(pic_ctx* c, SpeciesDev& s, int64_t* spilled) {
    const int ntile = c->g.nt[0] * c->g.nt[1] * c->g.nt[2];
    std::vector<int> h_count(ntile), h_holes(ntile);
    Counters h_ctr;
    if (cudaMemcpyAsync(h_count.data(), s.count, sizeof(int) * ntile, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return -1;
    if (cudaMemcpyAsync(h_holes.data(), s.holes, sizeof(int) * ntile, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return -1;
    if (cudaMemcpyAsync(&h_ctr, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return -1;
    int64_t n = 0;
    for (int t = 0; t < ntile; ++t) n += std::min(h_count[t], s.h_cap[t]) - h_holes[t];
    const int nsp = std::min(h_ctr.spill_count[c->step & 1], s.spill_cap);
    if (spilled) *spilled = nsp;
    return n + nsp;
}

// ---------------------------------------------------------------------------
// Fields: FP64 compact host layout <-> padded working-precision device arrays.

template <typename T>
__global__ void k_unpack(Geom g, const double* src, T* a0, T* a1, T* a2) {
    const long long N = g.host_N();
    const int nxs = g.n[0] + g.open_x;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % nxs), j = (int)((e / nxs) % g.n[1]), k = (int)(e / ((long long)nxs * g.n[1]));
        const T v0 = src ? (T)src[e] : T(0), v1 = src ? (T)src[N + e] : T(0), v2 = src ? (T)src[2 * N + e] : T(0);
        store3(g, a0, a1, a2, i, j, k, v0, v1, v2);
    }
}

template <typename T, typename A>
__global__ void k_pack(Geom g, const T* E0, const T* E1, const T* E2, const T* B0, const T* B1, const T* B2,
                       const A* J0, const A* J1, const A* J2, double jscale, double* E,
                       double* B, double* J) {
    const long long N = g.host_N();
    const int nxs = g.n[0] + g.open_x;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % nxs), j = (int)((e / nxs) % g.n[1]), k = (int)(e / ((long long)nxs * g.n[1]));
        const long long p = g.pidx(i, j, k);
        const long long cj = i < g.n[0] ? g.cidx(i, j, k) : -1;   // J has no slot on an open face
        if (E) {
            E[e] = (double)E0[p];
            E[N + e] = (double)E1[p];
            E[2 * N + e] = (double)E2[p];
        }
        if (B) {
            B[e] = (double)B0[p];
            B[N + e] = (double)B1[p];
            B[2 * N + e] = (double)B2[p];
        }
        if (J) {
            J[e] = cj < 0 ? 0.0 : (double)J0[cj] * jscale;
            J[N + e] = cj < 0 ? 0.0 : (double)J1[cj] * jscale;
            J[2 * N + e] = cj < 0 ? 0.0 : (double)J2[cj] * jscale;
        }
    }
}

template <typename T>
static pic_status unpack_t(pic_ctx* c, const double* E, const double* B) {
    LaunchScope ls(c, KC_OTHER);
    k_unpack<T><<<1024, 256, 0, c->stream>>>(c->g, E, (T*)c->E[0], (T*)c->E[1], (T*)c->E[2]);
    k_unpack<T><<<1024, 256, 0, c->stream>>>(c->g, B, (T*)c->B[0], (T*)c->B[1], (T*)c->B[2]);
    c->launches++;
    GBPIC_CHECK(c, cudaGetLastError());
    return PIC_OK;
}

pic_status unpack_fields(pic_ctx* c, const double* E, const double* B) {
    return c->prec == PIC_FP64 ? unpack_t<double>(c, E, B) : unpack_t<float>(c, E, B);
}

template <typename T>
static pic_status pack_t(pic_ctx* c, double* E, double* B, double* J) {
    LaunchScope ls(c, KC_OTHER);
    using A = typename JTraits<T>::acc_t;
    k_pack<T, A><<<1024, 256, 0, c->stream>>>(c->g, (T*)c->E[0], (T*)c->E[1], (T*)c->E[2], (T*)c->B[0], (T*)c->B[1],
                                               (T*)c->B[2], (const A*)c->J[0], (const A*)c->J[1], (const A*)c->J[2],
                                               c->jscale_J, E, B, J);
    GBPIC_CHECK(c, cudaGetLastError());
    return PIC_OK;
}

pic_status pack_fields(pic_ctx* c, double* E, double* B, double* J) {
    return c->prec == PIC_FP64 ? pack_t<double>(c, E, B, J) : pack_t<float>(c, E, B, J);
}

}  // namespace gbpic

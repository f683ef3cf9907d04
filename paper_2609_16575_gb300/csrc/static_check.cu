// pic_gauss_check_static: the Gauss-law check of pic_diagnostics (FP64 cloud-in-cell
// charge on the nodes, then max |div E - rho - rho_ion| and max |rho + rho_ion|) for
// callers that cannot allocate device memory.  pic_diagnostics allocates its node
// charge scratch on first use; this variant keeps that scratch in a file-scope static
// device array instead, so the call itself never allocates.
//
// Limits and sharing: the array holds the node charge of at most STATIC_MAX_CELLS
// cells plus two accumulators (8 MB); every GPU that loads the library holds it until
// the process exits.  All calls share it and it keeps the last call's contents, so
// each call clears what it uses first; calls whose work overlaps on the GPU (two
// contexts on different streams of one device, for instance) race on it.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <string>

#include "pic_internal.cuh"

namespace gbpic {

constexpr long long STATIC_MAX_CELLS = 1LL << 20;
constexpr int STATIC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_static_scratch[STATIC_MAX_CELLS + 32];

// Device address of g_static_scratch per device ordinal.  In host code the symbol
// name is only a host-side stand-in, so the address is looked up once per device
// (with that device current) and passed to the kernels.  The lookup loads this file's
// module on the device and commits the array, so it is done by pic_init_grid (which
// may allocate), not by the allocation-free entry point.
static std::atomic<double*> s_scratch[STATIC_MAX_DEVICES];

// Called by pic_init_grid with the context's device current.
pic_status static_scratch_prepare(pic_ctx* c) {
    const int dev = c->desc.device;
    if (dev < 0 || dev >= STATIC_MAX_DEVICES || s_scratch[dev].load()) return PIC_OK;
    double* p = nullptr;
    GBPIC_CHECK(c, cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_static_scratch));
    s_scratch[dev].store(p);
    return PIC_OK;
}

template <typename T>
__global__ void k_static_charge(Geom g, ParticleArrays<T> pa, const Rec<T>* spill, int nsp, double qdv, double* rho) {
    const int ntile = g.nt[0] * g.nt[1] * g.nt[2];
    auto one = [&](int gx, int gy, int gz, double dx, double dy, double dz, double w) {
        const double wx[2] = {1.0 - dx, dx}, wy[2] = {1.0 - dy, dy}, wz[2] = {1.0 - dz, dz};
        for (int c = 0; c < 2; ++c)
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    const int xx = x_after(g, gx + a);   // the face node of an open x has no slot
                    if (xx < 0) continue;
                    atomicAdd(rho + g.cidx(xx, wrap_idx(gy + b, g.n[1]), wrap_idx(gz + c, g.n[2])),
                              qdv * w * wx[a] * wy[b] * wz[c]);
                }
    };
    for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int cnt = min(pa.count[t], pa.cap[t]);
        const int tx = t % g.nt[0], ty = (t / g.nt[0]) % g.nt[1], tz = t / (g.nt[0] * g.nt[1]);
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const long long p = (long long)pa.seg_start[t] + i;
            const int lc = pa.cell[p];
            if (lc < 0) continue;
            one(tx * TILE + (lc & 7), ty * TILE + ((lc >> 3) & 7), tz * TILE + (lc >> 6), pa.d[0][p], pa.d[1][p],
                pa.d[2][p], pa.w[p]);
        }
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsp; i += gridDim.x * blockDim.x) {
        const Rec<T> r = spill[i];
        one(r.cell % g.n[0], (r.cell / g.n[0]) % g.n[1], r.cell / (g.n[0] * g.n[1]), r.d[0], r.d[1], r.d[2], r.w);
    }
}

template <typename T>
__global__ void k_static_gauss(Geom g, const T* E0, const T* E1, const T* E2, double d0, double d1, double d2,
                               double rho_ion, const double* rho, double* acc) {
    double mg = 0, mr = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.N; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % g.n[0]), j = (int)((e / g.n[0]) % g.n[1]), k = (int)(e / ((long long)g.n[0] * g.n[1]));
        const long long c = g.pidx(i, j, k), sy = g.Px, sz = (long long)g.Px * g.Gy;
        const double divE = ((double)E0[c] - (double)E0[c - 1]) / d0 + ((double)E1[c] - (double)E1[c - sy]) / d1 +
                            ((double)E2[c] - (double)E2[c - sz]) / d2;
        const double rt = rho[e] + rho_ion;
        mg = max_nf(mg, fabs(divE - rt));
        mr = max_nf(mr, fabs(rt));
    }
    for (int o = 16; o > 0; o >>= 1) {
        mg = fmax(mg, __shfl_xor_sync(0xffffffffu, mg, o));
        mr = fmax(mr, __shfl_xor_sync(0xffffffffu, mr, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(reinterpret_cast<unsigned long long*>(acc), (unsigned long long)__double_as_longlong(mg));
        atomicMax(reinterpret_cast<unsigned long long*>(acc + 1), (unsigned long long)__double_as_longlong(mr));
    }
}

template <typename T>
static pic_status gauss_static_t(pic_ctx* c, double* scratch, double* gauss_max, double* rho_max) {
    const Geom& g = c->g;
    double* rho = scratch;
    double* acc = scratch + STATIC_MAX_CELLS;
    GBPIC_CHECK(c, cudaMemsetAsync(rho, 0, sizeof(double) * (size_t)g.N, c->stream));
    GBPIC_CHECK(c, cudaMemsetAsync(acc, 0, sizeof(double) * 2, c->stream));
    const double* d = c->desc.d;
    const double dv = d[0] * d[1] * d[2];
    for (auto& s : c->species) {
        Counters h;
        GBPIC_CHECK(c, cudaMemcpyAsync(&h, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream));
        GBPIC_CHECK(c, cudaStreamSynchronize(c->stream));
        const int nsp = std::min(h.spill_count[c->step & 1], s.spill_cap);
        LaunchScope ls(c, KC_OTHER);
        k_static_charge<T><<<1024, 256, 0, c->stream>>>(g, arrays<T>(s), static_cast<const Rec<T>*>(s.spill), nsp,
                                                         s.q / dv, rho);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    {
        LaunchScope ls(c, KC_OTHER);
        k_static_gauss<T><<<1024, 256, 0, c->stream>>>(g, (const T*)c->E[0], (const T*)c->E[1], (const T*)c->E[2], d[0],
                                                        d[1], d[2], c->desc.rho_ion, rho, acc);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    double h[2];
    GBPIC_CHECK(c, cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    GBPIC_CHECK(c, cudaStreamSynchronize(c->stream));
    *gauss_max = h[0];
    *rho_max = h[1];
    return PIC_OK;
}

}  // namespace gbpic

using namespace gbpic;

extern "C" pic_status pic_gauss_check_static(pic_ctx* c, double* gauss_max, double* rho_max) {
    if (!c || !gauss_max || !rho_max) return PIC_ERR_ARG;
    if (c->g.N > STATIC_MAX_CELLS) {
        c->err = "pic_gauss_check_static: the grid has " + std::to_string(c->g.N) +
                 " cells, more than the static scratch maximum of " + std::to_string(STATIC_MAX_CELLS);
        return PIC_ERR_ARG;
    }
    const int dev = c->desc.device;
    if (dev < 0 || dev >= STATIC_MAX_DEVICES) return PIC_ERR_ARG;
    if (c->shape != PIC_SHAPE_CIC) {
        c->err = "pic_gauss_check_static: the CIC shape only";
        return PIC_ERR_STATE;
    }
    DeviceScope dscope_(dev);
    pic_status st = pic_sync(c);
    if (st != PIC_OK) return st;
    double* scratch = s_scratch[dev].load();
    if (!scratch) {
        c->err = "pic_gauss_check_static: the static scratch of this device was not set up by pic_init_grid";
        return PIC_ERR_STATE;
    }
    return c->prec == PIC_FP64 ? gauss_static_t<double>(c, scratch, gauss_max, rho_max)
                               : gauss_static_t<float>(c, scratch, gauss_max, rho_max);
}

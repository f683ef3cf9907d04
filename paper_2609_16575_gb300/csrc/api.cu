// C ABI of the library (include/gbpic.h): context set-up, the step loop of
// KEMPIC-3D section 2.2 (Fig. 2), read-out, diagnostics, timing and errors.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <tuple>

#include <nvtx3/nvToolsExt.h>
#include "pic_internal.cuh"

namespace gbpic {

void* dev_alloc(pic_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 256;
    void* p = nullptr;
    if (c->desc.alloc) {
        p = c->desc.alloc(bytes, c->desc.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->allocations.push_back(p);
    else c->err = "device allocation of " + std::to_string(bytes) + " bytes failed";
    return p;
}

cudaError_t raise_smem_limit(const void* kern, size_t bytes, int dev) {
    static std::mutex mu;
    static std::set<std::tuple<const void*, int, size_t>> done;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({kern, dev, bytes})) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done.insert({kern, dev, bytes});
    return e;
}

void dev_free(pic_ctx* c, void* p) {
    if (!p) return;
    auto it = std::find(c->allocations.begin(), c->allocations.end(), p);
    if (it != c->allocations.end()) c->allocations.erase(it);
    if (c->desc.alloc) c->desc.free(p, c->desc.alloc_user);
    else cudaFree(p);
}

pic_status cuda_fail(pic_ctx* c, cudaError_t e, const char* what) {
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return PIC_ERR_CUDA;
}

static cudaEvent_t take_event(pic_ctx* c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Kernel classes as named by pic_kernel_times and by the NVTX ranges around each launch
// (a profiler's timeline shows them; without one attached the ranges cost nothing).
static const char* const kKernelClassNames[KC_COUNT] = {"faraday_half", "tile_push", "list_push",   "append",
                                                        "ampere",       "sort",      "other",       "esk_crossers"};

void timing_begin(pic_ctx* c, int cls, cudaEvent_t* a) {
    nvtxRangePushA(kKernelClassNames[cls]);
    if (!c->timing) return;
    *a = take_event(c);
    cudaEventRecord(*a, c->stream);
}

void timing_end(pic_ctx* c, int cls, cudaEvent_t a) {
    nvtxRangePop();
    if (!c->timing || !a) return;
    cudaEvent_t b = take_event(c);
    cudaEventRecord(b, c->stream);
    c->pending.push_back({cls, a, b});
    // keep the number of outstanding events bounded
    if (c->pending.size() > 4096) {
        cudaEventSynchronize(c->pending.back().b);
        for (auto& p : c->pending) {
            float ms = 0;
            cudaEventElapsedTime(&ms, p.a, p.b);
            c->kc_ms[p.cls] += ms;
            c->kc_n[p.cls] += 1;
            c->event_pool.push_back(p.a);
            c->event_pool.push_back(p.b);
        }
        c->pending.clear();
    }
}

pic_status make_tensor_maps(pic_ctx* c) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    GBPIC_CHECK(c, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn) {
        c->err = "cuTensorMapEncodeTiled not available from the CUDA driver library";
        return PIC_ERR_CUDA;
    }
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    const Geom& g = c->g;
    const bool f64 = c->prec == PIC_FP64;
    const cuuint64_t es = f64 ? 8 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)g.n[0] + 2, (cuuint64_t)g.Gy, (cuuint64_t)g.Gz};
    cuuint64_t strides[2] = {(cuuint64_t)g.Px * es, (cuuint64_t)g.Px * g.Gy * es};
    cuuint32_t box[3] = {(cuuint32_t)(f64 ? Prec<double>::BX : Prec<float>::BX), (cuuint32_t)SB, (cuuint32_t)SB};
    cuuint32_t estr[3] = {1, 1, 1};
    for (int k = 0; k < 6; ++k) {
        void* base = k < 3 ? c->E[k] : c->B[k - 3];
        CUresult r = encode(&c->tmap[k], f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                            base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            c->err = "cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r);
            return PIC_ERR_CUDA;
        }
    }
    return PIC_OK;
}

static pic_status device_errors(pic_ctx* c) {
    int worst = 0;
    for (auto& s : c->species) {
        Counters h;
        GBPIC_CHECK(c, cudaMemcpy(&h, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost));
        worst |= h.err;
    }
    if (worst & ERRB_TIMEOUT) { c->err = "a bounded device wait for a TMA copy gave up"; return PIC_ERR_TIMEOUT; }
    if (worst & ERRB_OVERFLOW) { c->err = "mover or spill list overflow: particles were dropped"; return PIC_ERR_TILE_OVERFLOW; }
    // a non-finite momentum also makes its move look superluminal: report the cause
    if (worst & ERRB_NAN) { c->err = "non-finite momentum"; return PIC_ERR_NAN; }
    if (worst & ERRB_SUPERLUMINAL) { c->err = "a particle moved more than one cell in one step"; return PIC_ERR_SUPERLUMINAL; }
    return PIC_OK;
}

// The fixed-point unit of J (FP32 path): the coarsest unit any species, or the laser
// sheet (|J_y| <= 2 a0 / dx at one edge), needs; the FP64 path accumulates J itself.
void update_jscale(pic_ctx* c) {
    double js = 0;
    for (auto& s : c->species) js = std::max(js, s.jscale);
    if (c->laser_on) js = std::max(js, 2.0 * std::fabs(c->laser.a0) / c->desc.d[0] / std::ldexp(1.0, Prec<float>::JBITS));
    if (js <= 0 || c->prec == PIC_FP64) js = 1.0;
    c->jscale = js;
    c->jinv = 1.0 / js;
}

// One cycle of section 2.2, Fig. 2: Faraday half step, per species the tile push, the
// spill-list push, the mover append (and the periodic tile sort), Faraday half step,
// Ampere.  J is cleared by Ampere unless keep_j.  Expects J = 0 on entry.
bool window_moves_after(const pic_ctx* c, int64_t step) {
    if (!c->window_on) return false;
    const pic_window_desc& W = c->window;
    return step >= W.start && (step - W.start) % W.every == W.every - 1;
}

pic_status step_once(pic_ctx* c, double* rec, bool keep_j) {
    if (c->deposit == PIC_DEPOSIT_ESIRKEPOV && c->shape == PIC_SHAPE_CIC) {
        for (auto& s : c->species) {   // before the step changes anything
            const pic_status st = reserve_esk_records(c, s);
            if (st != PIC_OK) return st;
        }
    }
    c->jscale_J = c->jscale;
    const bool move = window_moves_after(c, c->step);
    pic_status st = launch_faraday_half(c, rec);
    if (st != PIC_OK) return st;
    for (size_t k = 0; k < c->species.size(); ++k) {
        st = launch_push_species(c, c->species[k], (int)(c->step & 1), rec ? rec + 2 : nullptr, move ? 1 : 0,
                                 move && (int)k == c->window.species);
        if (st != PIC_OK) return st;
    }
    st = launch_faraday_half(c, nullptr);
    if (st != PIC_OK) return st;
    if (c->filter_passes > 0) {
        st = launch_current_filter(c);         // the particles' J, before the laser sheet
        if (st != PIC_OK) return st;
    }
    if (c->g.open_x) {
        st = launch_open_x_before_ampere(c);   // laser sheet into J, face planes saved for Mur
        if (st != PIC_OK) return st;
    }
    st = launch_ampere(c, !keep_j);
    if (st != PIC_OK) return st;
    if (c->g.open_x) {
        st = launch_open_x_after_ampere(c);    // Mur condition on the two x faces
        if (st != PIC_OK) return st;
    }
    if (c->port_on || c->pec_y || c->pec_z) {
        st = launch_guide(c);                  // the port on x = 0, then the wall planes
        if (st != PIC_OK) return st;
    }
    if (move) {   // the end of the cycle: the window moves one cell along +x
        st = launch_window_shift(c);
        if (st != PIC_OK) return st;
        c->window_moves++;
    }
    c->step++;
    return PIC_OK;
}

}  // namespace gbpic

using namespace gbpic;

// Checkpoint / resume helpers (the blob layout of pic_save_state).
namespace gbpic {
pic_status load_species_ids(pic_ctx* c, const pic_species_desc* d, SpeciesDev& s, const double* ids);
}

namespace {
constexpr char kStateMagic[8] = {'G', 'B', 'P', 'I', 'C', 'S', 'T', '1'};
struct StateHeader {
    char magic[8];
    int32_t version, precision, n[3], bc_x, track_ids, nspecies;
    double d[3], dt;
    int64_t step, window_moves;
};
struct SpeciesHeader {
    double q, m, jscale;
    int64_t n_loaded, n_injected, escaped, rows;
};
template <typename V> void put(std::vector<unsigned char>& b, const V& v) {
    const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
    b.insert(b.end(), p, p + sizeof(V));
}
void put_doubles(std::vector<unsigned char>& b, const double* p, size_t n) {
    const unsigned char* q = reinterpret_cast<const unsigned char*>(p);
    b.insert(b.end(), q, q + n * sizeof(double));
}
}  // namespace

namespace gbpic {

pic_status run_as_graph(pic_ctx* c, const std::function<pic_status()>& body, bool* done) {
    *done = false;
    if (!c->capture_stream && cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        c->capture_stream = nullptr;
        return PIC_OK;
    }
    cudaStream_t run_stream = c->stream;
    c->stream = c->capture_stream;
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        ok = body() == PIC_OK;
        ok = cudaStreamEndCapture(c->stream, &graph) == cudaSuccess && ok;
    }
    c->stream = run_stream;
    cudaGraphExec_t exec = nullptr;
    ok = ok && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        c->err.clear();
        return PIC_OK;
    }
    const cudaError_t e = cudaGraphLaunch(exec, c->stream);
    cudaGraphExecDestroy(exec);   // freed once its launch completes
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
    *done = true;
    return PIC_OK;
}

}  // namespace gbpic

extern "C" {

const char* pic_status_string(pic_status s) {
    switch (s) {
        case PIC_OK: return "ok";
        case PIC_ERR_ARG: return "invalid argument";
        case PIC_ERR_CFL: return "time step violates the CFL condition";
        case PIC_ERR_OOM: return "device out of memory";
        case PIC_ERR_CUDA: return "CUDA error";
        case PIC_ERR_TILE_OVERFLOW: return "mover/spill overflow";
        case PIC_ERR_SUPERLUMINAL: return "particle moved more than one cell";
        case PIC_ERR_NAN: return "non-finite momentum";
        case PIC_ERR_STATE: return "call out of order";
        case PIC_ERR_TIMEOUT: return "device wait timed out";
        case PIC_ERR_NO_DEVICE: return "no sm_103 CUDA device";
    }
    return "unknown";
}

const char* pic_last_error(const pic_ctx* c) { return c ? c->err.c_str() : "null context"; }

int64_t pic_launch_count(const pic_ctx* c) { return c ? c->launches : 0; }

pic_status pic_init_grid(const pic_grid_desc* desc, pic_ctx** out) {
    if (!out) return PIC_ERR_ARG;
    *out = nullptr;
    if (!desc) return PIC_ERR_ARG;
    for (int k = 0; k < 3; ++k)
        if (desc->n[k] < 1 || !(desc->d[k] > 0) || !std::isfinite(desc->d[k])) return PIC_ERR_ARG;
    if (!(desc->dt > 0) || !std::isfinite(desc->dt)) return PIC_ERR_ARG;
    if (desc->precision != PIC_FP32 && desc->precision != PIC_FP64) return PIC_ERR_ARG;
    if (desc->alloc && !desc->free) return PIC_ERR_ARG;
    if ((long long)desc->n[0] * desc->n[1] * desc->n[2] > (1LL << 31) - 1) return PIC_ERR_ARG;
    if (desc->bc_x != 0 && desc->bc_x != 1) return PIC_ERR_ARG;
    if (desc->bc_x == 1 && desc->n[0] < 3) return PIC_ERR_ARG;
    // Eq. (15): c dt <= 1 / sqrt(sum 1/d^2)
    const double lim = 1.0 / std::sqrt(1.0 / (desc->d[0] * desc->d[0]) + 1.0 / (desc->d[1] * desc->d[1]) +
                                       1.0 / (desc->d[2] * desc->d[2]));
    if (desc->dt > lim * (1.0 + 1e-12)) return PIC_ERR_CFL;

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= desc->device || desc->device < 0) {
        cudaGetLastError();
        return PIC_ERR_NO_DEVICE;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, desc->device) != cudaSuccess || prop.major * 10 + prop.minor != 103)
        return PIC_ERR_NO_DEVICE;
    DeviceScope dscope_(desc->device);
    if (!dscope_.ok) return PIC_ERR_NO_DEVICE;

    pic_ctx* c = new (std::nothrow) pic_ctx();
    if (!c) return PIC_ERR_OOM;
    c->desc = *desc;
    c->prec = desc->precision;
    c->esize = c->prec == PIC_FP64 ? 8 : 4;
    Geom& g = c->g;
    for (int k = 0; k < 3; ++k) {
        g.n[k] = desc->n[k];
        g.nt[k] = (desc->n[k] + TILE - 1) / TILE;
    }
    g.Px = ((desc->n[0] + 2) + 7) / 8 * 8;
    g.Gy = desc->n[1] + 2;
    g.Gz = desc->n[2] + 2;
    g.N = (long long)desc->n[0] * desc->n[1] * desc->n[2];
    g.open_x = desc->bc_x == 1 ? 1 : 0;
    if (desc->stream) {
        c->stream = static_cast<cudaStream_t>(desc->stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return PIC_ERR_CUDA;
        }
        c->own_stream = true;
    }
    const size_t fb = (size_t)g.padded_size() * c->esize;
    for (int k = 0; k < 3; ++k) {
        c->E[k] = dev_alloc(c, fb);
        c->B[k] = dev_alloc(c, fb);
        c->J[k] = dev_alloc(c, sizeof(long long) * (size_t)g.N);   // int64 (FP32) or double (FP64)
        if (!c->E[k] || !c->B[k] || !c->J[k]) {
            pic_destroy(c);
            return PIC_ERR_OOM;
        }
        cudaMemsetAsync(c->E[k], 0, fb, c->stream);
        cudaMemsetAsync(c->B[k], 0, fb, c->stream);
        cudaMemsetAsync(c->J[k], 0, sizeof(long long) * (size_t)g.N, c->stream);
    }
    if (g.open_x) {
        c->mur_old = dev_alloc(c, (size_t)8 * desc->n[1] * desc->n[2] * c->esize);
        if (!c->mur_old) {
            pic_destroy(c);
            return PIC_ERR_OOM;
        }
    }
    if (desc->record_every > 0) {
        c->hist_cap = desc->history_capacity > 0 ? desc->history_capacity : 4096;
        c->hist = static_cast<double*>(dev_alloc(c, sizeof(double) * 3 * (size_t)c->hist_cap));
        if (!c->hist) {
            pic_destroy(c);
            return PIC_ERR_OOM;
        }
        cudaMemsetAsync(c->hist, 0, sizeof(double) * 3 * (size_t)c->hist_cap, c->stream);
    }
    pic_status st = make_tensor_maps(c);
    if (st == PIC_OK) st = static_scratch_prepare(c);
    if (st != PIC_OK) {
        std::fprintf(stderr, "gbpic: %s\n", c->err.c_str());
        pic_destroy(c);
        return st;
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        pic_destroy(c);
        return PIC_ERR_CUDA;
    }
    c->jscale = 1.0;
    c->jinv = 1.0;
    *out = c;
    return PIC_OK;
}

pic_status pic_set_fields(pic_ctx* c, const double* E, const double* B, int32_t device_pointers) {
    if (!c) return PIC_ERR_ARG;
    DeviceScope dscope_(c->desc.device);
    const size_t nb = sizeof(double) * 3 * (size_t)c->g.host_N();
    const double *dE = E, *dB = B;
    double* stage = nullptr;
    if (!device_pointers && (E || B)) {
        stage = static_cast<double*>(dev_alloc(c, 2 * nb));
        if (!stage) return PIC_ERR_OOM;
        if (E) GBPIC_CHECK(c, cudaMemcpyAsync(stage, E, nb, cudaMemcpyHostToDevice, c->stream));
        if (B) GBPIC_CHECK(c, cudaMemcpyAsync(stage + 3 * c->g.host_N(), B, nb, cudaMemcpyHostToDevice, c->stream));
        dE = E ? stage : nullptr;
        dB = B ? stage + 3 * c->g.host_N() : nullptr;
    }
    pic_status st = unpack_fields(c, dE, dB);
    GBPIC_CHECK(c, cudaStreamSynchronize(c->stream));
    if (stage) dev_free(c, stage);
    c->fields_set = true;
    c->gref_valid = false;
    c->rho_prev_step = -1;
    return st;
}

pic_status pic_load_species(pic_ctx* c, const pic_species_desc* d, int32_t* species_id) {
    if (!c || !d) return PIC_ERR_ARG;
    if (d->n < 0 || (d->n > 0 && (!d->X || !d->u || !d->w)) || !(d->m > 0) || !std::isfinite(d->q)) return PIC_ERR_ARG;
    if (d->mover_capacity < 0 || d->spill_capacity < 0) return PIC_ERR_ARG;
    if (c->pec_y || c->pec_z) {
        c->err = "pic_load_species: the conducting walls act on the fields only";
        return PIC_ERR_STATE;
    }
    DeviceScope dscope_(c->desc.device);
    c->species.emplace_back();
    SpeciesDev& s = c->species.back();
    pic_status st = load_species_impl(c, d, s);
    if (st != PIC_OK) {
        c->species.pop_back();
        return st;
    }
    if (!d->momenta_at_half_step && d->n > 0) {
        st = launch_backpush(c, s);
        if (st != PIC_OK) return st;
    }
    if (species_id) *species_id = (int32_t)c->species.size() - 1;
    c->gref_valid = false;
    c->rho_prev_step = -1;
    return PIC_OK;
}

// Whether the cycles of pic_step can run as a replayed two-cycle CUDA graph: nothing
// in a cycle's launches may depend on the step number beyond its parity (the particle
// blocks and the parity return to their state after two cycles), and no host work may
// come between cycles.  The laser, the port, the walls and the moving window change
// with time; the energy history and the per-kernel timing record host-side per cycle.
constexpr int GRAPH_MIN_PAIRS = 2;   // fewer pairs do not repay the capture
static bool graph_cycles(const pic_ctx* c) {
    return !c->timing && !c->hist && !c->g.open_x && !c->laser_on && !c->port_on && !c->pec_y && !c->pec_z &&
           !c->window_on && !c->species.empty();
}

// `pairs` pairs of cycles as one captured graph of two cycles, launched `pairs` times
// on the context's stream.  The capture runs on a stream of its own (the legacy default
// stream, torch's, cannot be captured; nothing runs while capturing, so the graph needs
// no link to it).  Capturing runs the host side of both cycles (step count, block
// parity), so each further launch advances the host state by two cycles as step_once
// would.  When the capture or the instantiation fails, the host state is put back and
// *done is false: the caller steps directly.
static pic_status step_pairs(pic_ctx* c, int pairs, bool* done) {
    *done = false;
    if (c->step_graph) {
        cudaGraphExecDestroy(c->step_graph);   // freed once its launches in flight complete
        c->step_graph = nullptr;
    }
    if (!c->capture_stream && cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        c->capture_stream = nullptr;
        return PIC_OK;
    }
    const int64_t launches0 = c->launches, step0 = c->step;
    std::vector<int> cur0;
    for (auto& sp : c->species) cur0.push_back(sp.cur);
    cudaStream_t run_stream = c->stream;
    c->stream = c->capture_stream;
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        ok = step_once(c, nullptr, false) == PIC_OK && step_once(c, nullptr, false) == PIC_OK;
        ok = cudaStreamEndCapture(c->stream, &graph) == cudaSuccess && ok;
    }
    c->stream = run_stream;
    ok = ok && graph && cudaGraphInstantiate(&c->step_graph, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        cudaGetLastError();
        if (c->step_graph) cudaGraphExecDestroy(c->step_graph);
        c->step_graph = nullptr;
        c->step = step0;
        c->launches = launches0;
        for (size_t i = 0; i < c->species.size(); ++i) c->species[i].cur = cur0[i];
        c->err.clear();
        return PIC_OK;
    }
    const int64_t per_pair = c->launches - launches0;
    for (int k = 0; k < pairs; ++k) {
        if (k > 0) {
            c->step += 2;
            c->launches += per_pair;
        }
        GBPIC_CHECK(c, cudaGraphLaunch(c->step_graph, c->stream));
    }
    *done = true;
    return PIC_OK;
}

pic_status pic_step(pic_ctx* c, int32_t nsteps) {
    if (!c || nsteps < 0) return PIC_ERR_ARG;
    if (nsteps == 0) return PIC_OK;
    if (c->window_on && c->window.species >= (int)c->species.size()) {
        c->err = "pic_step: the moving window's species is not loaded";
        return PIC_ERR_STATE;
    }
    DeviceScope dscope_(c->desc.device);
    update_jscale(c);
    if (c->j_dirty) {
        for (int k = 0; k < 3; ++k)
            GBPIC_CHECK(c, cudaMemsetAsync(c->J[k], 0, sizeof(long long) * (size_t)c->g.N, c->stream));
        c->j_dirty = false;
    }
    // launch-bound runs (many short cycles) save the launches' latency as a graph: the
    // first cycle runs directly (it makes any first-use allocation), the middle ones in
    // graph pairs, the last directly (it keeps J for pic_get_fields)
    const int pairs = graph_cycles(c) && nsteps >= 2 + 2 * GRAPH_MIN_PAIRS ? (nsteps - 2) / 2 : 0;
    for (int s = 0; s < nsteps; ++s) {
        if (s == 1 && pairs > 0) {
            bool done = false;
            const pic_status st = step_pairs(c, pairs, &done);
            if (st != PIC_OK) return st;
            if (done) {
                s += 2 * pairs - 1;
                continue;
            }
        }
        double* rec = nullptr;
        if (c->hist && c->step % c->desc.record_every == 0) {
            rec = c->hist + 3 * (c->hist_written % c->hist_cap);
            GBPIC_CHECK(c, cudaMemsetAsync(rec, 0, sizeof(double) * 3, c->stream));
            c->hist_written++;
        }
        pic_status st = step_once(c, rec, s == nsteps - 1);
        if (st != PIC_OK) return st;
    }
    c->j_dirty = true;
    return PIC_OK;
}

pic_status pic_set_laser(pic_ctx* c, const pic_laser_desc* laser) {
    if (!c) return PIC_ERR_ARG;
    if (!c->g.open_x) {
        c->err = "pic_set_laser needs an open x (bc_x = 1)";
        return PIC_ERR_STATE;
    }
    if (!laser) {
        c->laser_on = false;
        update_jscale(c);
        return PIC_OK;
    }
    if (laser->plane < 1 || laser->plane > c->g.n[0] - 1 || !(laser->tau > 0) || !(laser->w0 > 0) ||
        !std::isfinite(laser->a0) || !std::isfinite(laser->omega) || !std::isfinite(laser->t_peak))
        return PIC_ERR_ARG;
    c->laser = *laser;
    c->laser_on = true;
    update_jscale(c);
    return PIC_OK;
}

pic_status pic_set_moving_window(pic_ctx* c, const pic_window_desc* w) {
    if (!c) return PIC_ERR_ARG;
    if (!c->g.open_x) {
        c->err = "pic_set_moving_window needs an open x (bc_x = 1)";
        return PIC_ERR_STATE;
    }
    if (c->step != 0) {
        c->err = "pic_set_moving_window must precede stepping";
        return PIC_ERR_STATE;
    }
    if (!w) {
        c->window_on = false;
        return PIC_OK;
    }
    if (w->start < 0 || w->every < 1 || w->species < 0 || !(w->density > 0) || !std::isfinite(w->density) ||
        !std::isfinite(w->x0) || !(w->ramp >= 0) || !std::isfinite(w->ramp)) {
        c->err = "pic_set_moving_window: start >= 0, every >= 1, species >= 0, density > 0, ramp >= 0";
        return PIC_ERR_ARG;
    }
    long long ppc = 1;
    for (int k = 0; k < 3; ++k) {
        if (w->ppc[k] < 1) return PIC_ERR_ARG;
        ppc *= w->ppc[k];
    }
    if (w->ppc[0] > MAX_WINDOW_PPCX || ppc > 4096) {
        c->err = "pic_set_moving_window: ppc[0] <= 64 and ppc[0] ppc[1] ppc[2] <= 4096";
        return PIC_ERR_ARG;
    }
    if (w->species < (int)c->species.size()) {
        c->err = "pic_set_moving_window must precede loading the species it fills";
        return PIC_ERR_STATE;
    }
    c->window = *w;
    c->window_on = true;
    return PIC_OK;
}

int64_t pic_window_moves(const pic_ctx* c) { return c ? c->window_moves : 0; }

pic_status pic_set_background(pic_ctx* c, double rho_ion) {
    if (!c || !std::isfinite(rho_ion)) return PIC_ERR_ARG;
    c->desc.rho_ion = rho_ion;
    c->gref_valid = false;   // the Gauss reference includes the background
    return PIC_OK;
}

pic_status pic_set_pec(pic_ctx* c, int32_t pec_y, int32_t pec_z) {
    if (!c) return PIC_ERR_ARG;
    if ((pec_y != 0 && pec_y != 1) || (pec_z != 0 && pec_z != 1)) return PIC_ERR_ARG;
    if ((pec_y || pec_z) && !c->species.empty()) {
        c->err = "pic_set_pec: the conducting walls act on the fields only (species are loaded)";
        return PIC_ERR_STATE;
    }
    if ((pec_y || pec_z) && c->shape != PIC_SHAPE_CIC) {
        c->err = "pic_set_pec: the TSC shape supports a periodic box only";
        return PIC_ERR_STATE;
    }
    c->pec_y = pec_y;
    c->pec_z = pec_z;
    return PIC_OK;
}

pic_status pic_set_port(pic_ctx* c, const pic_port_desc* p) {
    if (!c) return PIC_ERR_ARG;
    if (!c->g.open_x) {
        c->err = "pic_set_port needs an open x (bc_x = 1)";
        return PIC_ERR_STATE;
    }
    if (!p) {
        c->port_on = false;
        return PIC_OK;
    }
    if (!(p->tau > 0) || p->mode_y < 1 || !std::isfinite(p->e0) || !std::isfinite(p->omega) || !std::isfinite(p->tau)) {
        c->err = "pic_set_port: tau > 0, mode_y >= 1, finite e0 and omega";
        return PIC_ERR_ARG;
    }
    c->port = *p;
    c->port_on = true;
    return PIC_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint / resume: the dynamical state as a host byte blob.


static pic_status save_state_impl(pic_ctx* c, void** blob, size_t* bytes);
static pic_status load_state_impl(pic_ctx* c, const void* blob, size_t bytes);

pic_status pic_save_state(pic_ctx* c, void** blob, size_t* bytes) {
    if (!c) return PIC_ERR_ARG;
    DeviceScope dscope_(c->desc.device);
    try {
        return save_state_impl(c, blob, bytes);
    } catch (const std::bad_alloc&) {
        return PIC_ERR_OOM;   // host memory for the blob
    }
}

pic_status pic_load_state(pic_ctx* c, const void* blob, size_t bytes) {
    if (!c) return PIC_ERR_ARG;
    DeviceScope dscope_(c->desc.device);
    try {
        return load_state_impl(c, blob, bytes);
    } catch (const std::bad_alloc&) {
        return PIC_ERR_OOM;
    }
}

static pic_status save_state_impl(pic_ctx* c, void** blob, size_t* bytes) {
    if (!c || !blob || !bytes) return PIC_ERR_ARG;
    *blob = nullptr;
    *bytes = 0;
    pic_status st = pic_sync(c);
    if (st != PIC_OK) return st;
    std::vector<unsigned char> b;
    StateHeader h{};
    memcpy(h.magic, kStateMagic, 8);
    h.version = 1;
    h.precision = c->prec;
    for (int k = 0; k < 3; ++k) {
        h.n[k] = c->g.n[k];
        h.d[k] = c->desc.d[k];
    }
    h.bc_x = c->g.open_x;
    h.track_ids = c->desc.track_ids ? 1 : 0;
    h.nspecies = (int32_t)c->species.size();
    h.dt = c->desc.dt;
    h.step = c->step;
    h.window_moves = c->window_moves;
    put(b, h);
    for (int k = 0; k < h.nspecies; ++k) {
        SpeciesDev& s = c->species[k];
        int64_t rows = 0;
        st = pic_get_particles(c, k, nullptr, &rows, 0);
        if (st != PIC_OK) return st;
        std::vector<double> P((size_t)7 * rows);
        if (rows > 0) {
            st = pic_get_particles(c, k, P.data(), &rows, 0);
            if (st != PIC_OK) return st;
        }
        Counters ctr;
        GBPIC_CHECK(c, cudaMemcpy(&ctr, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost));
        // the particles held (removed ids read as NaN and are left out; with ids each
        // keeps its own)
        std::vector<int64_t> keep;
        for (int64_t p = 0; p < rows; ++p)
            if (std::isfinite(P[(size_t)6 * rows + p])) keep.push_back(p);
        SpeciesHeader sh{s.q, s.m, s.jscale, s.n_loaded, s.n_injected, (int64_t)ctr.escaped, (int64_t)keep.size()};
        put(b, sh);
        std::vector<double> col(keep.size());
        for (int r = 0; r < 7; ++r) {
            for (size_t i = 0; i < keep.size(); ++i) col[i] = P[(size_t)r * rows + keep[i]];
            put_doubles(b, col.data(), col.size());
        }
        if (h.track_ids) {
            for (size_t i = 0; i < keep.size(); ++i) col[i] = (double)keep[i];
            put_doubles(b, col.data(), col.size());
        }
    }
    const size_t NH = (size_t)c->g.host_N();
    std::vector<double> E(3 * NH), B(3 * NH);
    st = pic_get_fields(c, E.data(), B.data(), nullptr, 0);
    if (st != PIC_OK) return st;
    put_doubles(b, E.data(), E.size());
    put_doubles(b, B.data(), B.size());
    void* out = std::malloc(b.size());
    if (!out) return PIC_ERR_OOM;
    memcpy(out, b.data(), b.size());
    *blob = out;
    *bytes = b.size();
    return PIC_OK;
}

void pic_free_state(void* blob) { std::free(blob); }

static pic_status load_state_impl(pic_ctx* c, const void* blob, size_t bytes) {
    if (!c || !blob || bytes < sizeof(StateHeader)) return PIC_ERR_ARG;
    StateHeader h;
    memcpy(&h, blob, sizeof(h));
    bool same = memcmp(h.magic, kStateMagic, 8) == 0 && h.version == 1 && h.precision == c->prec &&
                h.bc_x == c->g.open_x && h.track_ids == (c->desc.track_ids ? 1 : 0) && h.dt == c->desc.dt;
    for (int k = 0; k < 3; ++k) same = same && h.n[k] == c->g.n[k] && h.d[k] == c->desc.d[k];
    if (!same) {
        c->err = "pic_load_state: the state was saved from a context of another grid, precision or ids setting";
        return PIC_ERR_ARG;
    }
    if (!c->species.empty() || c->step != 0) {
        c->err = "pic_load_state needs a fresh context (no species loaded, no steps taken)";
        return PIC_ERR_STATE;
    }
    const unsigned char* p = static_cast<const unsigned char*>(blob) + sizeof(h);
    const unsigned char* end = static_cast<const unsigned char*>(blob) + bytes;
    auto take = [&](size_t n) -> const unsigned char* {
        if ((size_t)(end - p) < n) return nullptr;
        const unsigned char* q = p;
        p += n;
        return q;
    };
    struct Sp {
        SpeciesHeader sh;
        std::vector<double> cols;   // 7 rows (+ ids)
    };
    // counts bounded by what the blob can hold before any allocation or size arithmetic
    if (h.nspecies < 0 || (size_t)h.nspecies > bytes / sizeof(SpeciesHeader)) {
        c->err = "pic_load_state: malformed state";
        return PIC_ERR_ARG;
    }
    std::vector<Sp> sps(h.nspecies);
    for (auto& sp : sps) {
        const unsigned char* q = take(sizeof(SpeciesHeader));
        if (!q) return PIC_ERR_ARG;
        memcpy(&sp.sh, q, sizeof(SpeciesHeader));
        if (sp.sh.rows < 0 || (uint64_t)sp.sh.rows > bytes / (7 * sizeof(double))) {
            c->err = "pic_load_state: malformed state";
            return PIC_ERR_ARG;
        }
        const size_t nv = (size_t)sp.sh.rows * (h.track_ids ? 8 : 7);
        q = take(nv * sizeof(double));
        if (!q) return PIC_ERR_ARG;
        sp.cols.resize(nv);
        memcpy(sp.cols.data(), q, nv * sizeof(double));
    }
    const size_t NH = (size_t)c->g.host_N();
    const unsigned char* qe = take(3 * NH * sizeof(double));
    const unsigned char* qb = take(3 * NH * sizeof(double));
    if (!qe || !qb || p != end) {
        c->err = "pic_load_state: truncated or malformed state";
        return PIC_ERR_ARG;
    }
    std::vector<double> E(3 * NH), B(3 * NH);
    memcpy(E.data(), qe, E.size() * sizeof(double));
    memcpy(B.data(), qb, B.size() * sizeof(double));
    pic_status st = pic_set_fields(c, E.data(), B.data(), 0);
    if (st != PIC_OK) return st;
    DeviceScope dscope_(c->desc.device);
    for (auto& sp : sps) {
        const int64_t n = sp.sh.rows;
        std::vector<double> X(3 * (size_t)n), U(3 * (size_t)n), W((size_t)n);
        memcpy(X.data(), sp.cols.data(), 3 * n * sizeof(double));
        memcpy(U.data(), sp.cols.data() + 3 * n, 3 * n * sizeof(double));
        memcpy(W.data(), sp.cols.data() + 6 * n, n * sizeof(double));
        pic_species_desc d{};
        d.q = sp.sh.q;
        d.m = sp.sh.m;
        d.n = n;
        d.X = X.data();
        d.u = U.data();
        d.w = W.data();
        d.momenta_at_half_step = 1;
        c->species.emplace_back();
        SpeciesDev& s = c->species.back();
        st = load_species_ids(c, &d, s, h.track_ids ? sp.cols.data() + 7 * n : nullptr);
        if (st != PIC_OK) {
            c->species.pop_back();
            return st;
        }
        s.n_loaded = sp.sh.n_loaded;
        s.n_injected = sp.sh.n_injected;
        s.jscale = sp.sh.jscale;   // the fixed-point unit of J, as before
        const int escaped = (int)sp.sh.escaped;
        GBPIC_CHECK(c, cudaMemcpy(reinterpret_cast<char*>(s.ctr) + offsetof(Counters, escaped), &escaped, sizeof(int),
                                  cudaMemcpyHostToDevice));
    }
    c->step = h.step;
    c->window_moves = h.window_moves;
    c->gref_valid = false;
    c->rho_prev_step = -1;
    update_jscale(c);
    return PIC_OK;
}

pic_status pic_set_deposit(pic_ctx* c, int32_t deposit) {
    if (!c) return PIC_ERR_ARG;
    if (deposit != PIC_DEPOSIT_ZIGZAG && deposit != PIC_DEPOSIT_ESIRKEPOV) {
        c->err = "pic_set_deposit: PIC_DEPOSIT_ZIGZAG or PIC_DEPOSIT_ESIRKEPOV";
        return PIC_ERR_ARG;
    }
    c->deposit = deposit;
    return PIC_OK;
}

pic_status pic_set_shape(pic_ctx* c, int32_t shape) {
    if (!c) return PIC_ERR_ARG;
    if (shape != PIC_SHAPE_CIC && shape != PIC_SHAPE_TSC) {
        c->err = "pic_set_shape: PIC_SHAPE_CIC or PIC_SHAPE_TSC";
        return PIC_ERR_ARG;
    }
    if (shape == PIC_SHAPE_TSC && (c->g.open_x || c->pec_y || c->pec_z)) {
        c->err = "pic_set_shape: the TSC shape needs a periodic box without conducting walls";
        return PIC_ERR_STATE;
    }
    c->shape = shape;
    c->gref_valid = false;        // the Gauss reference and the continuity check use the
    c->rho_prev_step = -1;        // charge of the shape
    return PIC_OK;
}

pic_status pic_set_current_filter(pic_ctx* c, int32_t passes, int32_t compensate) {
    if (!c) return PIC_ERR_ARG;
    if (passes < 0 || passes > MAX_FILTER_PASSES || (compensate != 0 && compensate != 1)) {
        c->err = "pic_set_current_filter: 0 <= passes <= 8, compensate 0 or 1";
        return PIC_ERR_ARG;
    }
    c->filter_passes = passes;
    c->filter_compensate = passes > 0 ? compensate : 0;
    // the per-dimension kernel: `passes` binomial stencils, then the compensator
    double cur[2 * MAX_FILTER_PASSES + 3] = {1.0}, nxt[2 * MAX_FILTER_PASSES + 3];
    int len = 1;
    const double b[3] = {0.25, 0.5, 0.25};
    const double q[3] = {-passes / 4.0, 1.0 + passes / 2.0, -passes / 4.0};
    const int stages = passes + c->filter_compensate;
    for (int st = 0; st < stages; ++st) {
        const double* sten = st < passes ? b : q;
        for (int i = 0; i < len + 2; ++i) nxt[i] = 0.0;
        for (int i = 0; i < len; ++i)
            for (int m = 0; m < 3; ++m) nxt[i + m] += cur[i] * sten[m];
        len += 2;
        for (int i = 0; i < len; ++i) cur[i] = nxt[i];
    }
    for (int i = 0; i < len; ++i) c->filter_K[i] = cur[i];
    c->filter_h = (len - 1) / 2;
    return PIC_OK;
}

pic_status pic_set_wait_limit(pic_ctx* c, int32_t polls) {
    if (!c) return PIC_ERR_ARG;
    c->wait_polls = polls < 0 ? -1 : polls;
    return PIC_OK;
}

pic_status pic_sync(pic_ctx* c) {
    if (!c) return PIC_ERR_ARG;
    DeviceScope dscope_(c->desc.device);
    GBPIC_CHECK(c, cudaStreamSynchronize(c->stream));
    return device_errors(c);
}

pic_status pic_get_fields(pic_ctx* c, double* E, double* B, double* J, int32_t device_pointers) {
    if (!c) return PIC_ERR_ARG;
    DeviceScope dscope_(c->desc.device);
    pic_status st = pic_sync(c);
    if (st != PIC_OK && st != PIC_ERR_TILE_OVERFLOW) return st;
    const size_t nb = sizeof(double) * 3 * (size_t)c->g.host_N();
    if (device_pointers) {
        st = pack_fields(c, E, B, J);
        if (st != PIC_OK) return st;
        GBPIC_CHECK(c, cudaStreamSynchronize(c->stream));
        return PIC_OK;
    }
    double* stage = static_cast<double*>(dev_alloc(c, 3 * nb));
    if (!stage) return PIC_ERR_OOM;
    double* sE = E ? stage : nullptr;
    double* sB = B ? stage + 3 * c->g.host_N() : nullptr;
    double* sJ = J ? stage + 6 * c->g.host_N() : nullptr;
    if (J && !c->j_dirty) GBPIC_CHECK(c, cudaMemsetAsync(sJ, 0, nb, c->stream));
    st = pack_fields(c, sE, sB, c->j_dirty ? sJ : nullptr);
    if (st != PIC_OK) return st;
    if (E) GBPIC_CHECK(c, cudaMemcpyAsync(E, sE, nb, cudaMemcpyDeviceToHost, c->stream));
    if (B) GBPIC_CHECK(c, cudaMemcpyAsync(B, sB, nb, cudaMemcpyDeviceToHost, c->stream));
    if (J) GBPIC_CHECK(c, cudaMemcpyAsync(J, sJ, nb, cudaMemcpyDeviceToHost, c->stream));
    GBPIC_CHECK(c, cudaStreamSynchronize(c->stream));
    dev_free(c, stage);
    return PIC_OK;
}

pic_status pic_get_particles(pic_ctx* c, int32_t species, double* out, int64_t* n, int32_t device_pointers) {
    if (!c || !n || species < 0 || species >= (int32_t)c->species.size()) return PIC_ERR_ARG;
    DeviceScope dscope_(c->desc.device);
    pic_status st = pic_sync(c);
    if (st != PIC_OK && st != PIC_ERR_TILE_OVERFLOW) return st;
    SpeciesDev& s = c->species[species];
    int64_t alive = c->desc.track_ids ? s.n_loaded + s.n_injected : count_alive(c, s, nullptr);
    if (alive < 0) return cuda_fail(c, cudaGetLastError(), "count_alive");
    *n = alive;
    if (!out || alive == 0) return PIC_OK;
    const size_t nb = sizeof(double) * 7 * (size_t)alive;
    double* dst = out;
    if (!device_pointers) {
        dst = static_cast<double*>(dev_alloc(c, nb));
        if (!dst) return PIC_ERR_OOM;
    }
    if (c->desc.track_ids) GBPIC_CHECK(c, cudaMemsetAsync(dst, 0xff, nb, c->stream));   // NaN for lost ids
    st = get_particles_impl(c, s, dst, alive);
    if (st != PIC_OK) return st;
    if (!device_pointers) {
        GBPIC_CHECK(c, cudaMemcpy(out, dst, nb, cudaMemcpyDeviceToHost));
        dev_free(c, dst);
    }
    return PIC_OK;
}

pic_status pic_diagnostics(pic_ctx* c, pic_diag* out) {
    if (!c || !out) return PIC_ERR_ARG;
    DeviceScope dscope_(c->desc.device);
    pic_status st = pic_sync(c);
    if (st != PIC_OK) return st;
    return diagnostics_impl(c, out);
}

pic_status pic_get_history(pic_ctx* c, double* out, int32_t max_records, int32_t* count) {
    if (!c || !count) return PIC_ERR_ARG;
    DeviceScope dscope_(c->desc.device);
    *count = 0;
    if (!c->hist) return PIC_OK;
    GBPIC_CHECK(c, cudaStreamSynchronize(c->stream));
    const int64_t have = std::min<int64_t>(c->hist_written, c->hist_cap);
    const int64_t first = c->hist_written - have;
    std::vector<double> h(3 * (size_t)c->hist_cap);
    GBPIC_CHECK(c, cudaMemcpy(h.data(), c->hist, sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
    int32_t k = 0;
    for (int64_t r = first; r < c->hist_written && k < max_records; ++r, ++k) {
        const int64_t slot = r % c->hist_cap;
        if (out) memcpy(out + 3 * k, h.data() + 3 * slot, sizeof(double) * 3);
    }
    *count = k;
    return PIC_OK;
}

pic_status pic_set_timing(pic_ctx* c, int32_t enable) {
    if (!c) return PIC_ERR_ARG;
    DeviceScope dscope_(c->desc.device);
    GBPIC_CHECK(c, cudaStreamSynchronize(c->stream));
    c->timing = enable != 0;
    return PIC_OK;
}

pic_status pic_kernel_times(pic_ctx* c, int32_t max, const char** names, int64_t* launches, double* ms, int32_t* count) {
    const char* const* kNames = kKernelClassNames;
    if (!c || !count) return PIC_ERR_ARG;
    DeviceScope dscope_(c->desc.device);
    GBPIC_CHECK(c, cudaStreamSynchronize(c->stream));
    for (auto& p : c->pending) {
        float t = 0;
        cudaEventElapsedTime(&t, p.a, p.b);
        c->kc_ms[p.cls] += t;
        c->kc_n[p.cls] += 1;
        c->event_pool.push_back(p.a);
        c->event_pool.push_back(p.b);
    }
    c->pending.clear();
    int k = 0;
    for (int i = 0; i < KC_COUNT && k < max; ++i, ++k) {
        if (names) names[k] = kNames[i];
        if (launches) launches[k] = c->kc_n[i];
        if (ms) ms[k] = c->kc_ms[i];
    }
    *count = k;
    for (int i = 0; i < KC_COUNT; ++i) {
        c->kc_ms[i] = 0;
        c->kc_n[i] = 0;
    }
    return PIC_OK;
}

void pic_destroy(pic_ctx* c) {
    if (!c) return;
    DeviceScope dscope_(c->desc.device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->step_graph) cudaGraphExecDestroy(c->step_graph);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    adjoint_free(c);
    for (auto& p : c->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c->event_pool) cudaEventDestroy(e);
    std::vector<void*> all = c->allocations;
    for (void* p : all) dev_free(c, p);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"

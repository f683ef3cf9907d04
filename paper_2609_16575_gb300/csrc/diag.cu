// FP64 device reductions of the diagnostics of KEMPIC-3D section 3.3: field energy
// U_EM = 1/2 dV sum (E^n^2 + B^n^2), kinetic energy, the Gauss residual of Eq. (2)
// with CIC charge on the nodes, and the discrete continuity residual of Eq. (12).
// Whatever the working precision, these sums and the charge deposit run in FP64.
#include <cmath>
#include <cstring>
#include <limits>

#include "pic_internal.cuh"

namespace gbpic {

// accumulator layout in ctx->dacc (doubles): sums then maxima (stored as bit patterns
// of non-negative doubles so that atomicMax on 64-bit integers orders them)
enum { S_UE = 0, S_UB, S_K, M_GAUSS, M_GCHANGE, M_RHO, M_CONT, M_J, DACC_N };

__device__ __forceinline__ void acc_max(double* acc, int slot, double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(reinterpret_cast<unsigned long long*>(acc + slot), (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ void acc_sum(double* acc, int slot, double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(acc + slot, v);
}

template <typename T>
__global__ void k_energy(Geom g, Fields<T> f, double hx, double hy, double hz, double half_dv, double* acc) {
    double se = 0, sb = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.N; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % g.n[0]), j = (int)((e / g.n[0]) % g.n[1]), k = (int)(e / ((long long)g.n[0] * g.n[1]));
        const long long c = g.pidx(i, j, k), sy = g.Px, sz = (long long)g.Px * g.Gy;
        const double ex = f.E[0][c], ey = f.E[1][c], ez = f.E[2][c];
        // B^n = B^{n-1/2} - dt/2 curl E^n (Eq. (13) with a half step)
        const double bx = f.B[0][c] - (hy * ((double)f.E[2][c + sy] - ez) - hz * ((double)f.E[1][c + sz] - ey));
        const double by = f.B[1][c] - (hz * ((double)f.E[0][c + sz] - ex) - hx * ((double)f.E[2][c + 1] - ez));
        const double bz = f.B[2][c] - (hx * ((double)f.E[1][c + 1] - ey) - hy * ((double)f.E[0][c + sy] - ex));
        se += ex * ex + ey * ey + ez * ez;
        sb += bx * bx + by * by + bz * bz;
        if (g.open_x && i == g.n[0] - 1) {   // the face x = n: Ey, Ez and Bx live there
            const long long q = g.pidx(i + 1, j, k);
            const double eyf = f.E[1][q], ezf = f.E[2][q];
            const double bxf = f.B[0][q] - (hy * ((double)f.E[2][q + sy] - ezf) - hz * ((double)f.E[1][q + sz] - eyf));
            se += eyf * eyf + ezf * ezf;
            sb += bxf * bxf;
        }
    }
    acc_sum(acc, S_UE, se * half_dv);
    acc_sum(acc, S_UB, sb * half_dv);
}

// Node weights of the quadratic (TSC) shape for in-cell offset d: the nodes m - 1 ..
// m + 1 around the nearest node m (0 or 1), first node returned.
__device__ __forceinline__ int tsc_node_weights(double d, double w[3]) {
    const int m = d >= 0.5 ? 1 : 0;
    const double e = d - m, a = 0.5 - e, b = 0.5 + e;
    w[0] = 0.5 * a * a;
    w[1] = 0.75 - e * e;
    w[2] = 0.5 * b * b;
    return m - 1;
}

// Kinetic energy at u^{n-1/2} and the FP64 charge of the nodes with the particle
// shape: CIC (shape 1) or TSC (shape 2, periodic box).
template <typename T>
__global__ void k_particles(Geom g, ParticleArrays<T> pa, const Rec<T>* spill, int nsp, double q, double m,
                            double qdv, double* rho, double* acc, int shape) {
    const int ntile = g.nt[0] * g.nt[1] * g.nt[2];
    double ks = 0;
    auto one = [&](int gx, int gy, int gz, double dx, double dy, double dz, double ux, double uy, double uz, double w) {
        const double u2 = ux * ux + uy * uy + uz * uz;
        ks += w * m * (u2 / (sqrt(1.0 + u2) + 1.0));
        if (shape == 2) {
            double tx[3], ty[3], tz[3];
            const int bx = gx + tsc_node_weights(dx, tx), by = gy + tsc_node_weights(dy, ty),
                      bz = gz + tsc_node_weights(dz, tz);
            for (int c = 0; c < 3; ++c)
                for (int b = 0; b < 3; ++b)
                    for (int a = 0; a < 3; ++a) {
                        const long long e = g.cidx(wrap_idx(bx + a, g.n[0]), wrap_idx(by + b, g.n[1]), wrap_idx(bz + c, g.n[2]));
                        atomicAdd(rho + e, qdv * w * tx[a] * ty[b] * tz[c]);
                    }
            return;
        }
        const double wx[2] = {1.0 - dx, dx}, wy[2] = {1.0 - dy, dy}, wz[2] = {1.0 - dz, dz};
        for (int c = 0; c < 2; ++c)
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    const int xx = x_after(g, gx + a);   // the face node of an open x has no slot
                    if (xx < 0) continue;
                    const long long e = g.cidx(xx, wrap_idx(gy + b, g.n[1]), wrap_idx(gz + c, g.n[2]));
                    atomicAdd(rho + e, qdv * w * wx[a] * wy[b] * wz[c]);
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
                pa.d[2][p], pa.u[0][p], pa.u[1][p], pa.u[2][p], pa.w[p]);
        }
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsp; i += gridDim.x * blockDim.x) {
        const Rec<T> r = spill[i];
        one(r.cell % g.n[0], (r.cell / g.n[0]) % g.n[1], r.cell / (g.n[0] * g.n[1]), r.d[0], r.d[1], r.d[2], r.u[0],
            r.u[1], r.u[2], r.w);
    }
    acc_sum(acc, S_K, ks);
}

// Node residuals: Gauss G = div E - rho - rho_ion, its change from the reference,
// and continuity R = (rho - rho_prev)/dt + div J.
template <typename T>
__global__ void k_nodes(Geom g, Fields<T> f, const double* d, double rho_ion, double dt, double jscale,
                        const double* rho, double* rho_prev, double* gref, int gref_valid, int cont_valid, double* acc) {
    double mg = 0, mgc = 0, mr = 0, mc = 0, mj = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.N; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % g.n[0]), j = (int)((e / g.n[0]) % g.n[1]), k = (int)(e / ((long long)g.n[0] * g.n[1]));
        const long long c = g.pidx(i, j, k), sy = g.Px, sz = (long long)g.Px * g.Gy;
        const double divE = ((double)f.E[0][c] - (double)f.E[0][c - 1]) / d[0] +
                            ((double)f.E[1][c] - (double)f.E[1][c - sy]) / d[1] +
                            ((double)f.E[2][c] - (double)f.E[2][c - sz]) / d[2];
        const double rt = rho[e] + rho_ion;
        const double G = divE - rt;
        mg = max_nf(mg, fabs(G));
        mr = max_nf(mr, fabs(rt));
        if (gref_valid) mgc = max_nf(mgc, fabs(G - gref[e]));
        else gref[e] = G;
        // an open x has no edge left of node 0: its Jx there is zero
        const long long ex = (g.open_x && i == 0) ? -1 : g.cidx(wrap_idx(i - 1, g.n[0]), j, k);
        const long long ey = g.cidx(i, wrap_idx(j - 1, g.n[1]), k);
        const long long ez = g.cidx(i, j, wrap_idx(k - 1, g.n[2]));
        const double jx = (double)f.J[0][e] * jscale, jy = (double)f.J[1][e] * jscale, jz = (double)f.J[2][e] * jscale;
        mj = max_nf(mj, fmax(fabs(jx), fmax(fabs(jy), fabs(jz))));
        if (cont_valid) {
            const double jxm = ex < 0 ? 0.0 : (double)f.J[0][ex] * jscale;
            const double divJ = (jx - jxm) / d[0] + (jy - (double)f.J[1][ey] * jscale) / d[1] +
                                (jz - (double)f.J[2][ez] * jscale) / d[2];
            mc = max_nf(mc, fabs((rho[e] - rho_prev[e]) / dt + divJ));
        }
        rho_prev[e] = rho[e];
    }
    acc_max(acc, M_GAUSS, mg);
    acc_max(acc, M_GCHANGE, mgc);
    acc_max(acc, M_RHO, mr);
    acc_max(acc, M_CONT, mc);
    acc_max(acc, M_J, mj);
}

template <typename T>
static pic_status diag_t(pic_ctx* c, pic_diag* out) {
    const Geom& g = c->g;
    const size_t nb = sizeof(double) * (size_t)g.N;
    if (!c->rho) {
        c->rho = static_cast<double*>(dev_alloc(c, nb));
        c->rho_prev = static_cast<double*>(dev_alloc(c, nb));
        c->gref = static_cast<double*>(dev_alloc(c, nb));
        if (!c->rho || !c->rho_prev || !c->gref) return PIC_ERR_OOM;
    }
    if (!c->dacc) {
        c->dacc = static_cast<double*>(dev_alloc(c, sizeof(double) * (DACC_N + 3)));
        if (!c->dacc) return PIC_ERR_OOM;
    }
    double* dd = c->dacc + DACC_N;   // the cell sizes, for k_nodes
    GBPIC_CHECK(c, cudaMemsetAsync(c->dacc, 0, sizeof(double) * DACC_N, c->stream));
    GBPIC_CHECK(c, cudaMemcpyAsync(dd, c->desc.d, sizeof(double) * 3, cudaMemcpyHostToDevice, c->stream));
    GBPIC_CHECK(c, cudaMemsetAsync(c->rho, 0, nb, c->stream));
    Fields<T> f;
    for (int k = 0; k < 3; ++k) {
        f.E[k] = static_cast<T*>(c->E[k]);
        f.B[k] = static_cast<T*>(c->B[k]);
        f.J[k] = static_cast<typename JTraits<T>::acc_t*>(c->J[k]);
    }
    const double dt = c->desc.dt;
    const double* d = c->desc.d;
    const double dv = d[0] * d[1] * d[2];
    {
        LaunchScope ls(c, KC_OTHER);
        k_energy<T><<<1024, 256, 0, c->stream>>>(g, f, 0.5 * dt / d[0], 0.5 * dt / d[1], 0.5 * dt / d[2], 0.5 * dv, c->dacc);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    int64_t alive = 0, spilled = 0;
    for (auto& s : c->species) {
        int64_t sp = 0;
        const int64_t a = count_alive(c, s, &sp);
        if (a < 0) return cuda_fail(c, cudaGetLastError(), "count_alive");
        alive += a;
        spilled += sp;
        LaunchScope ls(c, KC_OTHER);
        k_particles<T><<<1024, 256, 0, c->stream>>>(g, arrays<T>(s), static_cast<const Rec<T>*>(s.spill), (int)sp, s.q,
                                                     s.m, s.q / dv, c->rho, c->dacc, c->shape);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    // a window move changes the frame: no continuity check across it, and the Gauss
    // reference is taken again
    const int cont_valid = (c->rho_prev_step >= 0 && c->step == c->rho_prev_step + 1 && c->j_dirty &&
                            c->window_moves_at_rho == c->window_moves) ? 1 : 0;
    if (c->gref_valid && c->window_moves_at_gref != c->window_moves) c->gref_valid = false;
    {
        LaunchScope ls(c, KC_OTHER);
        k_nodes<T><<<1024, 256, 0, c->stream>>>(g, f, dd, c->desc.rho_ion, dt, c->jscale_J, c->rho, c->rho_prev, c->gref,
                                                 c->gref_valid ? 1 : 0, cont_valid, c->dacc);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    double h[DACC_N];
    GBPIC_CHECK(c, cudaMemcpyAsync(h, c->dacc, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    GBPIC_CHECK(c, cudaStreamSynchronize(c->stream));
    out->step = c->step;
    out->t = c->step * dt;
    out->U_E = h[S_UE];
    out->U_B = h[S_UB];
    out->K_half = h[S_K];
    out->gauss_max = h[M_GAUSS];
    out->gauss_change_max = c->gref_valid ? h[M_GCHANGE] : 0.0;
    out->rho_max = h[M_RHO];
    out->cont_max = cont_valid ? h[M_CONT] : std::numeric_limits<double>::quiet_NaN();
    out->J_max = c->j_dirty ? h[M_J] : 0.0;
    out->n_alive = alive;
    out->n_spilled = spilled;
    out->n_escaped = 0;
    for (auto& s : c->species) {
        Counters h;
        GBPIC_CHECK(c, cudaMemcpy(&h, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost));
        out->n_escaped += h.escaped;
    }
    if (!c->gref_valid) c->window_moves_at_gref = c->window_moves;
    c->gref_valid = true;
    c->rho_prev_step = c->step;
    c->window_moves_at_rho = c->window_moves;
    return PIC_OK;
}

// U_E = 1/2 dV sum E^n^2 and U_B = 1/2 dV sum B^n^2 of the current state (FP64).
template <typename T>
static pic_status energy_t(pic_ctx* c, double* UE, double* UB) {
    if (!c->dacc) {
        c->dacc = static_cast<double*>(dev_alloc(c, sizeof(double) * (DACC_N + 3)));
        if (!c->dacc) return PIC_ERR_OOM;
    }
    GBPIC_CHECK(c, cudaMemsetAsync(c->dacc, 0, sizeof(double) * DACC_N, c->stream));
    Fields<T> f;
    for (int k = 0; k < 3; ++k) {
        f.E[k] = static_cast<T*>(c->E[k]);
        f.B[k] = static_cast<T*>(c->B[k]);
        f.J[k] = nullptr;
    }
    const double dt = c->desc.dt;
    const double* d = c->desc.d;
    {
        LaunchScope ls(c, KC_OTHER);
        k_energy<T><<<1024, 256, 0, c->stream>>>(c->g, f, 0.5 * dt / d[0], 0.5 * dt / d[1], 0.5 * dt / d[2],
                                                  0.5 * d[0] * d[1] * d[2], c->dacc);
        GBPIC_CHECK(c, cudaGetLastError());
    }
    double h[2];
    GBPIC_CHECK(c, cudaMemcpyAsync(h, c->dacc, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    GBPIC_CHECK(c, cudaStreamSynchronize(c->stream));
    *UE = h[S_UE];
    *UB = h[S_UB];
    return PIC_OK;
}

pic_status energy_sums(pic_ctx* c, double* UE, double* UB) {
    return c->prec == PIC_FP64 ? energy_t<double>(c, UE, UB) : energy_t<float>(c, UE, UB);
}

pic_status diagnostics_impl(pic_ctx* c, pic_diag* out) {
    return c->prec == PIC_FP64 ? diag_t<double>(c, out) : diag_t<float>(c, out);
}

}  // namespace gbpic

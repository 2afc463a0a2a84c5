// Reverse mode of the 2D leapfrog recurrence: d L / d eps_r over a design
// rectangle for losses of the running DFT at monitor cells.
//
// The paper only remarks that message-passing layers are differentiable
// (Sec. IV-A); this is the discrete adjoint of Prop. 2's two layers: the
// transposed layers in reverse order.  With the adjoint state (e, hx, hy, psi)
// holding dL/d(state) after a step, one reverse step is
//   layer 2 transposed:  gx = (Cb/dx)(1 + cEx) e + cEx psi_ezx,
//                        gy = -(Cb/dy)(1 + cEy) e + cEy psi_ezy,
//                        hy(i) += gx(i) - gx(i+1),  hx(j) += gy(j) - gy(j+1),
//                        psi_ezx <- bEx (psi_ezx + (Cb/dx) e),
//                        psi_ezy <- bEy (psi_ezy - (Cb/dy) e),  e <- Ca e;
//   layer 1 transposed:  fx = Db_x (1 + cHx) hy + cHx psi_hyx,
//                        fy = -Db_y (1 + cHy) hx + cHy psi_hxy,
//                        e(i,j) += fy(j-1) - fy(j) + fx(i-1) - fx(i),
//                        psi_hxy <- bHy (psi_hxy - Db_y hx), psi_hyx <- bHx (psi_hyx + Db_x hy),
// after dL/dE^{n+1} is added at the monitor cells.  The sweep stores e over the
// design cells for every step of a checkpoint segment; a reduction then forms
//   dL/deps_r += sum_n e (dCa/deps_r E^n + dCb/deps_r curlH^{n+1/2})
// from it and the recomputed forward values (no read-modify-write in the sweep).
//
// The kernel streams rows like the forward kernel: layer 2 transposed at row a
// reads row a+1 at the previous level (the same-iteration ring slot), layer 1
// transposed reads row a-1 at the same level (previous iteration), so the same
// skewed wavefront applies T reverse steps per HBM pass.  gy of the row above
// is produced at the end of the previous level (no second coefficient lookup);
// the general variant keeps fy of the row below in a per-level register ring
// because that row's psi_hxy has already moved on.  Three variants run side by
// side on their own streams: CPML strips, strips near the design, adjoint
// sources or the ragged edge (no CPML state), and clean interior strips.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <type_traits>
#include <vector>

#include "gem_internal.h"

namespace gem {

int step_prepare(fdtd_ctx* c, int64_t n_steps);

namespace {

constexpr int A_PF_G = 3;
constexpr int A_Q_I = 8;

// Stage slots per lane and row: interior e hx hy; lite adds the design band's
// Ca, Cb/dx, Cb/dy; CPML adds the four psi and, after the material words, the
// row's y-profile scalars.  pv = CPML variant.
__host__ __device__ constexpr int a_nslot(bool gen, bool pv) { return pv ? 7 : (gen ? 6 : 3); }
__host__ __device__ constexpr int a_stage_f4(bool gen, bool pv, int groups = 1) {
    return a_nslot(gen, pv) * 32 + 8 + (pv ? groups : 0);
}
__host__ __device__ constexpr int a_stages(int T, bool pv) { return pv ? T + A_PF_G : A_Q_I; }
__host__ __device__ constexpr int a_pf(int T, bool pv) { return pv ? A_PF_G : A_Q_I - T; }

size_t adj_smem(int T, int warps, bool gen, bool pv, int groups = 1) {
    return (size_t)warps * a_stages(T, pv) * a_stage_f4(gen, pv, groups) * sizeof(float4);
}

__device__ __forceinline__ void acp16(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void acp4(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void acommit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void await_() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ float& cref(float4& v, int c) { return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w)); }
__device__ __forceinline__ float cget(const float4& v, int c) { return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w)); }

// Adjoint source entry of a task: cell (i, j) gets adj_src[n * n_adj + slot].
// Reuses Sample2 {i, j, comp (unused), slot}.

// GEN: design rectangle, adjoint sources, ragged edge; PMLV: CPML auxiliaries
// One warp's reverse task (or, G < 32, 32 / G narrow tasks of G lanes each, one
// per lane group, as in the forward general task: width-G shuffles, every group
// streams as many rows as the warp's longest task and stores nothing past its
// own, adjoint sources read from memory).  coef_s: the scene's coefficient
// table, float4 (Ca, Cb/dx, Cb/dy, Cb) or, for square cells, float2
// (Ca, Cb/dx) (Cb/dy is then the same float); stage0: the warp's staging area.
template <int T, bool GEN, bool PMLV, bool DSGV = true, int G = 32, typename CT = float4>
__device__ __forceinline__ void adj_task(const TmzDev* __restrict__ S, const Task& tk,
                                         const Sample2* __restrict__ srcs, int parity, long long n_top,
                                         const CT* coef_s, float4* stage0, int lane) {
    static_assert(G == 32 || (GEN && PMLV && G >= 4 && G < 32 && (G & (G - 1)) == 0), "narrow groups are CPML tasks");
    constexpr bool PV = GEN && PMLV;
    constexpr bool SD = GEN && !PMLV;   // design band staged
    constexpr int Q = a_stages(T, PV);
    constexpr int PF = a_pf(T, PV);
    constexpr int SF4 = a_stage_f4(GEN, PV, 32 / G);
    constexpr int NS = a_nslot(GEN, PV);
    const int pitch = S->pitch, nx = S->nx, ny = S->ny;
    const float* __restrict__ e_in = S->f[F_EZ][parity];
    const float* __restrict__ hx_in = S->f[F_HX][parity];
    const float* __restrict__ hy_in = S->f[F_HY][parity];
    float* __restrict__ e_out = S->f[F_EZ][parity ^ 1];
    float* __restrict__ hx_out = S->f[F_HX][parity ^ 1];
    float* __restrict__ hy_out = S->f[F_HY][parity ^ 1];
    const uint8_t* __restrict__ mat = S->mat;
    const float dbx = S->dbx, dby = S->dby;

    const int gl = lane & (G - 1);             // lane within the task's group
    const int grp = lane / G;
    const int cx = tk.x0 - HALO + 4 * gl;
    const int cs = cx + PAD_X;
    const bool out_lane = (gl >= HALO / 4) && (gl < G - HALO / 4) && (cx < nx) && (tk.xe == 0 || cx < tk.xe) &&
                          !(tk.flags & TASK_NOSTORE);
    const int s_row = tk.ya - T;
    const int r_last = tk.yb + T - 1;
    int n_iter = r_last - s_row + 1;
    if constexpr (G < 32) n_iter = (int)__reduce_max_sync(0xffffffffu, (unsigned)n_iter);

    const bool pml = PV && (tk.flags & TASK_PML) != 0;
    const bool dsg = GEN && DSGV && (tk.flags & TASK_DSG) != 0;   // DSGV = false: built without design code
    const bool has_src = GEN && tk.samp_end > tk.samp_begin;
    const int dsg_i0 = S->dsg_i0, dsg_j0 = S->dsg_j0, dsg_w = S->dsg_w, dsg_h = S->dsg_h;
    const float4* __restrict__ dsg_coef = S->dsg_coef;
    const float* __restrict__ band = S->dsg_band;
    const size_t band_plane = (size_t)dsg_h * pitch;
    const long long rec_n0 = S->dsg_rec_n0, rec_len = S->dsg_rec_len;
    float* const adj_rec = S->adj_rec;
    const int adj_edges = S->adj_edges;
    const float* __restrict__ adj_src = S->adj_src;
    const int n_adj = S->n_adj;
    // the task's adjoint source cells: the first 32 ride in lane registers
    const int n_samp = tk.samp_end - tk.samp_begin;
    Sample2 my_samp;
    my_samp.i = -1; my_samp.j = -1; my_samp.comp = 0; my_samp.slot = 0;
    if (GEN && G == 32 && lane < n_samp) my_samp = srcs[tk.samp_begin + lane];
    const int npml = S->has_pml;
    const float* pr = S->prof;
    const int prow = S->rows;
    bool lane_px = false;
    float bex[4] = {0, 0, 0, 0}, cex[4] = {0, 0, 0, 0}, bhx[4] = {0, 0, 0, 0}, chx[4] = {0, 0, 0, 0};
    if (PV && pml) {
        lane_px = (cx < npml) || (cx + 3 >= nx - npml);
        if (lane_px)
            for (int q = 0; q < 4; q++) {
                bex[q] = pr[cs + q];
                cex[q] = pr[pitch + cs + q];
                bhx[q] = pr[2 * pitch + cs + q];
                chx[q] = pr[3 * pitch + cs + q];
            }
    }
    float* psi_in[4] = {S->f[F_PEZX][parity], S->f[F_PEZY][parity], S->f[F_PHXY][parity], S->f[F_PHYX][parity]};
    float* psi_out[4] = {S->f[F_PEZX][parity ^ 1], S->f[F_PEZY][parity ^ 1], S->f[F_PHXY][parity ^ 1],
                         S->f[F_PHYX][parity ^ 1]};

    auto stage_of = [&](int row) { return stage0 + ((row - s_row) % Q) * SF4; };
    auto yslab = [&](int row) { return (row < npml) || (row >= ny - npml); };
    // stage the row of iteration i (past its last row, a group re-reads that row)
    auto issue = [&](int i) {
        const int row = G < 32 ? min(s_row + i, r_last) : s_row + i;
        float4* st = stage0 + (i % Q) * SF4;
        const size_t g = (size_t)(row + PAD_Y) * pitch + cs;
        acp16(st + 0 * 32 + lane, e_in + g);
        acp16(st + 1 * 32 + lane, hx_in + g);
        acp16(st + 2 * 32 + lane, hy_in + g);
        acp4(reinterpret_cast<uint32_t*>(st + NS * 32) + lane, mat + g);
        if constexpr (SD) {
            if (dsg && row >= dsg_j0 && row < dsg_j0 + dsg_h) {
                const float* b = band + (size_t)(row - dsg_j0) * pitch + cs;
                acp16(st + 3 * 32 + lane, b);
                acp16(st + 4 * 32 + lane, b + band_plane);
                acp16(st + 5 * 32 + lane, b + 2 * band_plane);
            }
        }
        if constexpr (PV) {
            if (pml) {
                // the row's bEy, cEy, bHy, cHy
                if (yslab(row) && gl < 4)
                    acp4(reinterpret_cast<float*>(st + NS * 32 + 8 + grp) + gl, pr + 4 * pitch + gl * prow + row + PAD_Y);
                if (lane_px) {
                    acp16(st + 3 * 32 + lane, psi_in[0] + g);
                    acp16(st + 6 * 32 + lane, psi_in[3] + g);
                }
                if (yslab(row)) {
                    acp16(st + 4 * 32 + lane, psi_in[1] + g);
                    acp16(st + 5 * 32 + lane, psi_in[2] + g);
                }
            }
        }
    };
    // coefficients of row `row` (material table, or the design override)
    auto coefs = [&](uint32_t m, int row, float4* c) {
        if constexpr (std::is_same<CT, float2>::value) {
            const float2 a0 = coef_s[m & 255u], a1 = coef_s[(m >> 8) & 255u];
            const float2 a2 = coef_s[(m >> 16) & 255u], a3 = coef_s[m >> 24];
            c[0] = make_float4(a0.x, a0.y, a0.y, 0.f);
            c[1] = make_float4(a1.x, a1.y, a1.y, 0.f);
            c[2] = make_float4(a2.x, a2.y, a2.y, 0.f);
            c[3] = make_float4(a3.x, a3.y, a3.y, 0.f);
        } else {
            c[0] = coef_s[m & 255u];
            c[1] = coef_s[(m >> 8) & 255u];
            c[2] = coef_s[(m >> 16) & 255u];
            c[3] = coef_s[m >> 24];
        }
        if constexpr (GEN) {
            if (dsg) {
                const int dj = row - dsg_j0;
                if (dj >= 0 && dj < dsg_h) {
                    if constexpr (SD) {
                        const float4* st = stage_of(row);
                        const float4 ca = st[3 * 32 + lane], cbx = st[4 * 32 + lane], cby = st[5 * 32 + lane];
                        c[0] = make_float4(ca.x, cbx.x, cby.x, 0.f);
                        c[1] = make_float4(ca.y, cbx.y, cby.y, 0.f);
                        c[2] = make_float4(ca.z, cbx.z, cby.z, 0.f);
                        c[3] = make_float4(ca.w, cbx.w, cby.w, 0.f);
                    } else {
                        const float4* drow = dsg_coef + (size_t)dj * dsg_w;
                        const int di = cx - dsg_i0;
                        for (int q = 0; q < 4; q++)
                            if (di + q >= 0 && di + q < dsg_w) c[q] = drow[di + q];
                    }
                }
            }
        }
    };
    // y-profile scalar k (bEy, cEy, bHy, cHy) of a CPML row, from its stage
    auto yp = [&](const float4* sta, int k) { return reinterpret_cast<const float*>(sta + NS * 32 + 8 + grp)[k]; };
    // gy of a row whose adjoint state is final for the level just finished
    auto gy_of = [&](const float4& e, const float4* c, int row, const float4* sta) {
        float4 g = make_float4(-c[0].z * e.x, -c[1].z * e.y, -c[2].z * e.z, -c[3].z * e.w);
        if constexpr (PV) {
            if (pml && yslab(row)) {
                const float ce = yp(sta, 1);
                const float4 p = sta[4 * 32 + lane];
                g.x = g.x * (1.f + ce) + ce * p.x;
                g.y = g.y * (1.f + ce) + ce * p.y;
                g.z = g.z * (1.f + ce) + ce * p.z;
                g.w = g.w * (1.f + ce) + ce * p.w;
            }
        }
        return g;
    };

    // add dL/dE^{m+1} (table row m) at the adjoint source cells of `row`; this
    // must precede every use of the row's state for reverse step m, including
    // the gy the row below takes from it
    auto inject = [&](float4& e, int row, long long m) {
        if constexpr (GEN) {
            if (has_src && m >= 0) {
                const int nq = G == 32 ? (n_samp < 32 ? n_samp : 32) : 0;   // groups read sources from memory
                for (int q = 0; q < nq; q++) {
                    if (__shfl_sync(0xffffffffu, my_samp.j, q) != row) continue;   // warp-uniform
                    const int d = __shfl_sync(0xffffffffu, my_samp.i, q) - cx;
                    const int slot = __shfl_sync(0xffffffffu, my_samp.slot, q);
                    if (d >= 0 && d < 4) cref(e, d) += adj_src[m * n_adj + slot];
                }
                for (int q = tk.samp_begin + (G == 32 ? 32 : 0); q < tk.samp_end; q++) {
                    const Sample2 sp = srcs[q];
                    const int d = sp.i - cx;
                    if (sp.j == row && d >= 0 && d < 4) cref(e, d) += adj_src[m * n_adj + sp.slot];
                }
            }
        }
    };

    float4 E[T + 1], X[T + 2], Y[T + 1], GY[T + 1], FY[T + 1];
    uint32_t M[T + 1];
#pragma unroll
    for (int k = 0; k < T + 1; k++) {
        E[k] = make_float4(0, 0, 0, 0);
        Y[k] = E[k];
        GY[k] = E[k];
        FY[k] = E[k];
        M[k] = 0;
    }
#pragma unroll
    for (int k = 0; k < T + 2; k++) X[k] = make_float4(0, 0, 0, 0);
#pragma unroll
    for (int k = 0; k < PF; k++) {
        issue(k);
        acommit();
    }

#pragma unroll 1
    for (int it = 0; it < n_iter; ++it) {
        const int r = s_row + it;
        await_<PF - 1>();
#pragma unroll
        for (int k = T + 1; k >= 1; k--) X[k] = X[k - 1];
#pragma unroll
        for (int k = T; k >= 1; k--) {
            E[k] = E[k - 1];
            Y[k] = Y[k - 1];
            M[k] = M[k - 1];
        }
        {
            const float4* st = stage_of(r);
            E[0] = st[0 * 32 + lane];
            X[0] = st[1 * 32 + lane];
            Y[0] = st[2 * 32 + lane];
            M[0] = reinterpret_cast<const uint32_t*>(st + NS * 32)[lane];
        }
        // level 1 reverses step n_top: the new row first gets dL/dE^{n_top+1},
        // then its gy for level 1 of the row below it
        inject(E[0], r, n_top);
        {
            float4 c[4];
            coefs(M[0], r, c);
            GY[0] = gy_of(E[0], c, r, stage_of(r));
        }

#pragma unroll
        for (int t = 1; t <= T; t++) {
            const int a = r - t;
            if constexpr (GEN) {
                if (a < s_row) continue;
            }
            const long long n = n_top - (t - 1);   // forward step being reversed
            float4* sta = stage_of(a);
            float4 c[4];
            coefs(M[t], a, c);
            // E[t] already holds dL/dE^{n+1} (added when the row's previous level
            // finished, or when it was loaded): dL/deps_r over owned design cells
            if constexpr (GEN) {
                if (dsg && a >= tk.ya && a < tk.yb && out_lane) {
                    // keep dL/dE^{n+1} of the owned design cells; a reduction after
                    // the segment forms dL/deps_r from it and the recorded E^n, curl H
                    const int dj = a - dsg_j0;
                    const long long nr = n - rec_n0;
                    if (dj >= 0 && dj < dsg_h && nr >= 0 && nr < rec_len) {
                        const size_t hw = (size_t)dsg_w * dsg_h;
                        float* er = adj_rec + (size_t)nr * hw * (adj_edges ? 3 : 1) + (size_t)dj * dsg_w;
                        const int di = cx - dsg_i0;
                        for (int q = 0; q < 4; q++) {
                            const int d = di + q;
                            if (d >= 0 && d < dsg_w) er[d] = cget(E[t], q);
                        }
                    }
                }
            }
            // ---- layer 2 transposed ----
            float4 gx = make_float4(c[0].y * E[t].x, c[1].y * E[t].y, c[2].y * E[t].z, c[3].y * E[t].w);   // (Cb/dx) e
            float4 ux = gx;
            float4 gya = make_float4(-c[0].z * E[t].x, -c[1].z * E[t].y, -c[2].z * E[t].z, -c[3].z * E[t].w);
            float4 uy = make_float4(-gya.x, -gya.y, -gya.z, -gya.w);                                      // (Cb/dy) e
            if constexpr (PV) {
                if (pml) {
                    if (lane_px) {
                        const float4 p = sta[3 * 32 + lane];
                        gx.x = gx.x * (1.f + cex[0]) + cex[0] * p.x;
                        gx.y = gx.y * (1.f + cex[1]) + cex[1] * p.y;
                        gx.z = gx.z * (1.f + cex[2]) + cex[2] * p.z;
                        gx.w = gx.w * (1.f + cex[3]) + cex[3] * p.w;
                    }
                    if (yslab(a)) {
                        const float ce = yp(sta, 1);
                        const float4 p = sta[4 * 32 + lane];
                        gya.x = gya.x * (1.f + ce) + ce * p.x;
                        gya.y = gya.y * (1.f + ce) + ce * p.y;
                        gya.z = gya.z * (1.f + ce) + ce * p.z;
                        gya.w = gya.w * (1.f + ce) + ce * p.w;
                    }
                }
            }
            const float gxr = __shfl_down_sync(0xffffffffu, gx.x, 1, G);
            Y[t].x += gx.x - gx.y;
            Y[t].y += gx.y - gx.z;
            Y[t].z += gx.z - gx.w;
            Y[t].w += gx.w - gxr;
            const float4 gyu = GY[t - 1];   // gy of row a+1 (final for level t-1)
            X[t].x += gya.x - gyu.x;
            X[t].y += gya.y - gyu.y;
            X[t].z += gya.z - gyu.z;
            X[t].w += gya.w - gyu.w;
            if constexpr (GEN) {
                // X[t], Y[t] now hold dL/dHx^{n+1/2}, dL/dHy^{n+1/2} of row a (the
                // next step's self-loop plus layer 2 transposed): keep them over the
                // owned design cells for the edge-weight gradients
                if (adj_edges && dsg && a >= tk.ya && a < tk.yb && out_lane) {
                    const int dj = a - dsg_j0;
                    const long long nr = n - rec_n0;
                    if (dj >= 0 && dj < dsg_h && nr >= 0 && nr < rec_len) {
                        const size_t hw = (size_t)dsg_w * dsg_h;
                        float* xr = adj_rec + ((size_t)nr * 3 + 1) * hw + (size_t)dj * dsg_w;
                        const int di = cx - dsg_i0;
                        for (int q = 0; q < 4; q++) {
                            const int d = di + q;
                            if (d >= 0 && d < dsg_w) {
                                xr[d] = cget(X[t], q);
                                xr[hw + d] = cget(Y[t], q);
                            }
                        }
                    }
                }
            }
            if constexpr (PV) {
                if (pml) {
                    if (lane_px) {
                        float4 p = sta[3 * 32 + lane];
                        p.x = bex[0] * (p.x + ux.x);
                        p.y = bex[1] * (p.y + ux.y);
                        p.z = bex[2] * (p.z + ux.z);
                        p.w = bex[3] * (p.w + ux.w);
                        sta[3 * 32 + lane] = p;
                    }
                    if (yslab(a)) {
                        const float be = yp(sta, 0);
                        float4 p = sta[4 * 32 + lane];
                        p.x = be * (p.x - uy.x);
                        p.y = be * (p.y - uy.y);
                        p.z = be * (p.z - uy.z);
                        p.w = be * (p.w - uy.w);
                        sta[4 * 32 + lane] = p;
                    }
                }
            }
            E[t].x *= c[0].x;
            E[t].y *= c[1].x;
            E[t].z *= c[2].x;
            E[t].w *= c[3].x;
            // ---- layer 1 transposed ----
            float4 fx = make_float4(dbx * Y[t].x, dbx * Y[t].y, dbx * Y[t].z, dbx * Y[t].w);
            float4 fya = make_float4(-dby * X[t].x, -dby * X[t].y, -dby * X[t].z, -dby * X[t].w);
            float4 fyd;   // fy of row a-1
            if constexpr (PV) {
                if (pml) {
                    if (lane_px) {
                        const float4 p = sta[6 * 32 + lane];
                        fx.x = fx.x * (1.f + chx[0]) + chx[0] * p.x;
                        fx.y = fx.y * (1.f + chx[1]) + chx[1] * p.y;
                        fx.z = fx.z * (1.f + chx[2]) + chx[2] * p.z;
                        fx.w = fx.w * (1.f + chx[3]) + chx[3] * p.w;
                    }
                    if (yslab(a)) {
                        const float ch = yp(sta, 3);
                        const float4 p = sta[5 * 32 + lane];
                        fya.x = fya.x * (1.f + ch) + ch * p.x;
                        fya.y = fya.y * (1.f + ch) + ch * p.y;
                        fya.z = fya.z * (1.f + ch) + ch * p.z;
                        fya.w = fya.w * (1.f + ch) + ch * p.w;
                    }
                }
                fyd = FY[t];
                FY[t] = fya;
            } else {
                fyd = make_float4(-dby * X[t + 1].x, -dby * X[t + 1].y, -dby * X[t + 1].z, -dby * X[t + 1].w);
            }
            const float fxl = __shfl_up_sync(0xffffffffu, fx.w, 1, G);
            E[t].x += fyd.x - fya.x + fxl - fx.x;
            E[t].y += fyd.y - fya.y + fx.x - fx.y;
            E[t].z += fyd.z - fya.z + fx.y - fx.z;
            E[t].w += fyd.w - fya.w + fx.z - fx.w;
            if constexpr (PV) {
                if (pml) {
                    if (yslab(a)) {
                        const float bh = yp(sta, 2);
                        float4 p = sta[5 * 32 + lane];
                        p.x = bh * (p.x - dby * X[t].x);
                        p.y = bh * (p.y - dby * X[t].y);
                        p.z = bh * (p.z - dby * X[t].z);
                        p.w = bh * (p.w - dby * X[t].w);
                        sta[5 * 32 + lane] = p;
                    }
                    if (lane_px) {
                        float4 p = sta[6 * 32 + lane];
                        p.x = bhx[0] * (p.x + dbx * Y[t].x);
                        p.y = bhx[1] * (p.y + dbx * Y[t].y);
                        p.z = bhx[2] * (p.z + dbx * Y[t].z);
                        p.w = bhx[3] * (p.w + dbx * Y[t].w);
                        sta[6 * 32 + lane] = p;
                    }
                }
            }
            // level t+1 reverses step n-1: add dL/dE^{n} to this row now, then form
            // its gy for level t+1 of the row below
            if (t < T) {
                inject(E[t], a, n - 1);
                GY[t] = gy_of(E[t], c, a, sta);
            }
        }

        const int o = r - T;
        if (o >= tk.ya && o < tk.yb) {
            const size_t g = (size_t)(o + PAD_Y) * pitch + cs;
            if (out_lane) {
                if (cx + 3 < nx) {
                    *reinterpret_cast<float4*>(e_out + g) = E[T];
                    *reinterpret_cast<float4*>(hx_out + g) = X[T];
                    *reinterpret_cast<float4*>(hy_out + g) = Y[T];
                } else {
                    for (int q = 0; q < 4 && cx + q < nx; q++) {
                        e_out[g + q] = cget(E[T], q);
                        hx_out[g + q] = cget(X[T], q);
                        hy_out[g + q] = cget(Y[T], q);
                    }
                }
                if constexpr (PV) {
                    if (pml) {
                        const float4* sto = stage_of(o);
                        for (int q = 0; q < 4 && cx + q < nx; q++) {
                            if (yslab(o)) {
                                psi_out[1][g + q] = cget(sto[4 * 32 + lane], q);
                                psi_out[2][g + q] = cget(sto[5 * 32 + lane], q);
                            }
                            if (lane_px) {
                                psi_out[0][g + q] = cget(sto[3 * 32 + lane], q);
                                psi_out[3][g + q] = cget(sto[6 * 32 + lane], q);
                            }
                        }
                    }
                }
            }
        }
        // rows past r_last stay inside the pad rows
        issue(it + PF);
        acommit();
    }
    await_<0>();
}

// SQ (interior tasks of square-cell scenes): the table staged as (Ca, Cb/dx)
template <int T, bool GEN, bool PMLV, bool DSGV = true, bool SQ = false>
__global__ void __launch_bounds__((GEN && !PMLV) ? 128 : 256, (GEN && PMLV) ? 1 : (GEN ? 3 : 2)) k_adj(const TmzDev* __restrict__ scenes,
                                                          const Task* __restrict__ tasks, int n_tasks,
                                                          const Sample2* __restrict__ srcs, int parity,
                                                          long long n_top) {
    constexpr bool PV = GEN && PMLV;
    constexpr int Q = a_stages(T, PV);
    constexpr int SF4 = a_stage_f4(GEN, PV);
    using CT = typename std::conditional<SQ, float2, float4>::type;
    extern __shared__ float4 smem_f4[];
    __shared__ CT coef_s[256];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int warps = blockDim.x >> 5;
    const int tid = blockIdx.x * warps + wib;
    const TmzDev* S = scenes + tasks[blockIdx.x * warps].scene;
    for (int k = threadIdx.x; k < 256; k += blockDim.x) {
        const float4 c = S->coef[k];
        if constexpr (SQ) coef_s[k] = make_float2(c.x, c.y);
        else coef_s[k] = c;
    }
    __syncthreads();
    if (tid >= n_tasks) return;
    const Task tk = tasks[tid];
    if (tk.scene < 0) return;
    adj_task<T, GEN, PMLV, DSGV, 32, CT>(S, tk, srcs, parity, n_top, coef_s, smem_f4 + (size_t)wib * Q * SF4, lane);
}

// the reverse sweep's CPML tasks without a design in reach, in one launch: the
// first nw_blocks CTAs run whole-warp tasks, the rest the narrow x-slab tasks,
// 32 / NG_LANES per warp (both lists padded to whole CTAs of one scene)
template <int T>
__global__ void __launch_bounds__(256, 1) k_adj_cpml_mixed(const TmzDev* __restrict__ scenes,
                                                          const Task* __restrict__ tasks_w, int nw_blocks,
                                                          const Task* __restrict__ tasks_n,
                                                          const Sample2* __restrict__ srcs, int parity,
                                                          long long n_top) {
    constexpr int Q = a_stages(T, true);
    constexpr int SF_W = a_stage_f4(true, true), SF_N = a_stage_f4(true, true, 32 / NG_LANES);
    constexpr int PER_WARP = 32 / NG_LANES;
    extern __shared__ float4 smem_f4[];
    __shared__ float4 coef_s[256];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int warps = blockDim.x >> 5;
    const bool narrow = (int)blockIdx.x >= nw_blocks;
    const Task* first = narrow ? tasks_n + (size_t)(blockIdx.x - nw_blocks) * warps * PER_WARP
                               : tasks_w + (size_t)blockIdx.x * warps;
    if (first->scene < 0) return;
    const TmzDev* S = scenes + first->scene;
    for (int k = threadIdx.x; k < 256; k += blockDim.x) coef_s[k] = S->coef[k];
    __syncthreads();
    if (!narrow) {
        const Task tk = tasks_w[(size_t)blockIdx.x * warps + wib];
        if (tk.scene < 0) return;
        adj_task<T, true, true, false>(S, tk, srcs, parity, n_top, coef_s, smem_f4 + (size_t)wib * Q * SF_W, lane);
    } else {
        const Task* tw = first + (size_t)wib * PER_WARP;
        if (tw[0].scene < 0) return;   // a padding warp (whole warps only)
        const Task tk = tw[lane / NG_LANES];
        adj_task<T, true, true, false, NG_LANES>(S, tk, srcs, parity, n_top, coef_s,
                                                 smem_f4 + (size_t)wib * Q * SF_N, lane);
    }
}

template <int T, bool GEN, bool PMLV, bool DSGV = true, bool SQ = false>
cudaError_t launch_adj_v(const TmzDev* dev, const Task* tasks, int n, int warps, const Sample2* srcs, int parity,
                         long long n_top, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const size_t sm = adj_smem(T, warps, GEN, GEN && PMLV);
    cudaError_t e = ensure_dyn_smem((const void*)k_adj<T, GEN, PMLV, DSGV, SQ>, sm);
    if (e != cudaSuccess) return e;
    k_adj<T, GEN, PMLV, DSGV, SQ><<<n / warps, warps * 32, sm, st>>>(dev, tasks, n, srcs, parity, n_top);
    return cudaGetLastError();
}

struct AdjLists {
    const Task *t0, *t1, *t2, *t3;   // interior, CPML without a design in reach, lite, CPML with one
    const Task* tn;                  // narrow x-slab CPML tasks (32 / NG_LANES per warp)
    int n0, n1, n2, n3, nn, w0, w1, w2;
    int sq;                          // every scene has square cells: interior tasks stage (Ca, Cb/dx)
};

template <int T>
cudaError_t launch_adj_mixed(const TmzDev* dev, const AdjLists& L, const Sample2* srcs, int parity, long long n_top,
                             cudaStream_t st) {
    const int warps = L.w1;
    const size_t sm = adj_smem(T, warps, true, true, 32 / NG_LANES);
    cudaError_t e = ensure_dyn_smem((const void*)k_adj_cpml_mixed<T>, sm);
    if (e != cudaSuccess) return e;
    const int nw = L.n1 / warps, nb = L.nn / (warps * 32 / NG_LANES);
    k_adj_cpml_mixed<T><<<nw + nb, warps * 32, sm, st>>>(dev, L.t1, nw, L.tn, srcs, parity, n_top);
    return cudaGetLastError();
}

template <int T>
cudaError_t launch_adj_T(const TmzDev* dev, const AdjLists& L, const Sample2* srcs, int parity, long long n_top,
                         cudaStream_t s0, cudaStream_t s1, cudaStream_t s2) {
    cudaError_t e = L.nn > 0 ? launch_adj_mixed<T>(dev, L, srcs, parity, n_top, s1)
                             : launch_adj_v<T, true, true, false>(dev, L.t1, L.n1, L.w1, srcs, parity, n_top, s1);
    if (e == cudaSuccess) e = launch_adj_v<T, true, true>(dev, L.t3, L.n3, L.w1, srcs, parity, n_top, s1);
    if (e == cudaSuccess) e = launch_adj_v<T, true, false>(dev, L.t2, L.n2, L.w2, srcs, parity, n_top, s2);
    if (e == cudaSuccess)
        e = L.sq ? launch_adj_v<T, false, false, true, true>(dev, L.t0, L.n0, L.w0, srcs, parity, n_top, s0)
                 : launch_adj_v<T, false, false>(dev, L.t0, L.n0, L.w0, srcs, parity, n_top, s0);
    return e;
}

// dL/deps_r += fac * sum over the segment's steps of e^{n+1} r^n
__global__ void k_grad_reduce(const float* __restrict__ rec, const float* __restrict__ erec,
                              const float* __restrict__ fac, float* __restrict__ grad, int hw, int len) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= hw) return;
    float g = 0.f;
    for (int s = 0; s < len; s++) g += erec[(size_t)s * hw + c] * rec[(size_t)s * hw + c];
    grad[c] += fac[c] * g;
}

// the fields of the window (i0 - 1 .. i0 + w) x (j0 - 1 .. j0 + h) around a design
// rectangle after one step: out[3][H][W] = Ez^{n+1}, Hx^{n+1/2}, Hy^{n+1/2}
__global__ void k_edge_record(const float* __restrict__ ez, const float* __restrict__ hx,
                              const float* __restrict__ hy, int pitch, int i0, int j0, int W, int H,
                              float* __restrict__ out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int ww = W * H;
    if (q >= ww) return;
    const int i = i0 - 1 + q % W, j = j0 - 1 + q / W;
    const size_t g = (size_t)(j + PAD_Y) * pitch + i + PAD_X;
    out[q] = ez[g];
    out[ww + q] = hx[g];
    out[2 * ww + q] = hy[g];
}

// dL/dw of the 11 edge classes of every design cell (the order of
// fdtd_edge_grad), summed over one segment: for layer 2 the destination's
// dL/dE^{n+1} times the source's value in E^n or H^{n+1/2}, for layer 1 the
// destination's dL/dH^{n+1/2} times the source's value in E^n or H^{n-1/2}.
// win: the segment's windows [len][3][h+2][w+2] (k_edge_record after step n);
// prev: the window after the step before the segment, NULL at step 0 (the
// fields start at zero); erec: [len][3][h*w] = dL/dE^{n+1}, dL/dHx^{n+1/2},
// dL/dHy^{n+1/2} kept by the adjoint kernels.
__global__ void k_edge_reduce(const float* __restrict__ win, const float* __restrict__ prev,
                              const float* __restrict__ erec, float* __restrict__ g, int w, int h, int len) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int hw = w * h;
    if (c >= hw) return;
    const int W = w + 2, ww = W * (h + 2);
    const int x = (c / w + 1) * W + c % w + 1;
    float a[11];
#pragma unroll
    for (int k = 0; k < 11; k++) a[k] = 0.f;
    for (int s = 0; s < len; s++) {
        const float* cur = win + (size_t)s * 3 * ww;
        const float* pv = s > 0 ? cur - (size_t)3 * ww : prev;
        float ez = 0.f, ez_n = 0.f, ez_e = 0.f, hx0 = 0.f, hy0 = 0.f;
        if (pv) {
            ez = pv[x];
            ez_n = pv[x + W];
            ez_e = pv[x + 1];
            hx0 = pv[ww + x];
            hy0 = pv[2 * ww + x];
        }
        const float hx1 = cur[ww + x], hx1_s = cur[ww + x - W];
        const float hy1 = cur[2 * ww + x], hy1_w = cur[2 * ww + x - 1];
        const float* lr = erec + (size_t)s * 3 * hw;
        const float le = lr[c], lx = lr[hw + c], ly = lr[2 * hw + c];
        a[0] += le * ez;
        a[1] += le * hy1;
        a[2] += le * hy1_w;
        a[3] += le * hx1;
        a[4] += le * hx1_s;
        a[5] += lx * hx0;
        a[6] += lx * ez_n;
        a[7] += lx * ez;
        a[8] += ly * hy0;
        a[9] += ly * ez_e;
        a[10] += ly * ez;
    }
#pragma unroll
    for (int k = 0; k < 11; k++) g[(size_t)k * hw + c] += a[k];
}

}  // namespace

// ---------------------------------------------------------------------------
// host: checkpoints and the reverse sweep
// ---------------------------------------------------------------------------
struct AdjState {
    int every;
    int store;                     // 1: history kept (no recompute); 0: field checkpoints
    int edges;                     // 1: the history is the field window of each design (edge weights)
    std::vector<float*> ckpt;      // [slot * n_scenes + scene] -> F_COUNT2 padded arrays
    std::vector<float*> hist;      // [slot * n_scenes + scene] -> every x design cells of r^n
};

static size_t field_bytes(const Scene2* s) { return (size_t)s->pitch * s->rows * sizeof(float); }
static size_t design_cells(const Scene2* s) { return s->d_dsg ? (size_t)s->dsg_w * s->dsg_h : 0; }
static size_t window_cells(const Scene2* s) { return s->d_dsg ? (size_t)(s->dsg_w + 2) * (s->dsg_h + 2) : 0; }
// every cell of the window around the design lies outside the CPML slabs and
// inside the stored grid, so the 11 edges of each design cell are all its edges
static bool window_inside(const Scene2* s) {
    const int m = s->npml;
    return s->dsg_i0 - 1 >= m && s->dsg_j0 - 1 >= m && s->dsg_i0 + s->dsg_w <= s->nx - 1 - m &&
           s->dsg_j0 + s->dsg_h <= s->ny - 1 - m;
}

// store mode: point every scene's recording at the history block of the
// segment that contains step t
static void patch_for_step(const fdtd_ctx* c, const AdjState* A, TmzDev* dev, int64_t t) {
    const int ns = (int)c->s2.size();
    const int64_t slot = t / A->every;
    for (int k = 0; k < ns; k++) {
        const size_t q = (size_t)slot * ns + k;
        float* h = q < A->hist.size() ? A->hist[q] : nullptr;
        dev[k].dsg_rec = h;
        dev[k].dsg_rec_n0 = slot * A->every;
        dev[k].dsg_rec_len = h ? A->every : 0;
    }
}

void adj_patch_descriptors(fdtd_ctx* c, TmzDev* dev) {
    const AdjState* A = (const AdjState*)c->adj;
    if (!A || A->every <= 0 || !A->store) return;
    patch_for_step(c, A, dev, c->t);
}

int adj_checkpoint_if_due(fdtd_ctx* c) {
    AdjState* A = (AdjState*)c->adj;
    if (!A || A->every <= 0 || c->t % A->every) return FDTD_OK;
    NvtxRange nvtx("checkpoint");
    const int slot = (int)(c->t / A->every);
    const int ns = (int)c->s2.size();
    if (A->store) {
        if ((int)A->hist.size() < (slot + 1) * ns) A->hist.resize((size_t)(slot + 1) * ns, nullptr);
        for (int k = 0; k < ns; k++) {
            const Scene2* s = c->s2[k];
            if (A->edges && s->d_dsg && !window_inside(s)) {
                c->err = "edge-weight gradients need the design rectangle and a ring of one cell around it "
                         "outside the CPML and inside the grid";
                return FDTD_EINVAL;
            }
            const size_t hw = A->edges ? 3 * window_cells(s) : design_cells(s);
            float*& p = A->hist[(size_t)slot * ns + k];
            if (hw && !p && cudaMalloc(&p, (size_t)A->every * hw * sizeof(float)) != cudaSuccess) {
                cudaGetLastError();
                p = nullptr;
                c->err = "design history: out of device memory (FDTD_OPT_ADJ_STORE = 0 recomputes instead)";
                return FDTD_ENOMEM;
            }
        }
        if ((int)c->h_scenes.size() != ns) return FDTD_OK;   // descriptors not built yet: rebuild patches them
        patch_for_step(c, A, c->h_scenes.data(), c->t);
        cudaError_t e = cudaMemcpyAsync(c->d_scenes, c->h_scenes.data(), ns * sizeof(TmzDev), cudaMemcpyHostToDevice,
                                        c->stream);
        if (e != cudaSuccess) {
            c->err = std::string("design history descriptors: ") + cudaGetErrorString(e);
            return FDTD_ECUDA;
        }
        return FDTD_OK;
    }
    if ((int)A->ckpt.size() < (slot + 1) * ns) A->ckpt.resize((size_t)(slot + 1) * ns, nullptr);
    for (int k = 0; k < ns; k++) {
        Scene2* s = c->s2[k];
        float*& p = A->ckpt[(size_t)slot * ns + k];
        const size_t fb = field_bytes(s);
        if (!p && cudaMalloc(&p, F_COUNT2 * fb) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            c->err = "checkpoint: out of device memory";
            return FDTD_ENOMEM;
        }
        for (int f = 0; f < F_COUNT2; f++) {
            cudaError_t e = cudaMemcpyAsync((char*)p + f * fb, s->fbuf[f][c->parity], fb, cudaMemcpyDeviceToDevice, c->stream);
            if (e != cudaSuccess) {
                c->err = std::string("checkpoint copy: ") + cudaGetErrorString(e);
                return FDTD_ECUDA;
            }
        }
    }
    return FDTD_OK;
}

bool adj_edge_mode(const fdtd_ctx* c) {
    const AdjState* A = (const AdjState*)c->adj;
    return A && A->every > 0 && A->edges;
}

// the fused kernels keep the window themselves; the unfused pair (one step per
// call) has it copied out after each step
int adj_edge_record(fdtd_ctx* c, int steps_done) {
    const AdjState* A = (const AdjState*)c->adj;
    const int ns = (int)c->s2.size();
    // the step just taken is c->t + steps_done - 1 (single steps in this mode)
    const int64_t n = c->t + steps_done - 1;
    const int64_t slot = n / A->every, step_in = n % A->every;
    for (int k = 0; k < ns; k++) {
        const Scene2* s = c->s2[k];
        const size_t q = (size_t)slot * ns + k;
        if (!s->d_dsg || q >= A->hist.size() || !A->hist[q]) continue;
        const int W = s->dsg_w + 2, H = s->dsg_h + 2;
        float* out = A->hist[q] + (size_t)step_in * 3 * W * H;
        k_edge_record<<<(W * H + 255) / 256, 256, 0, c->stream>>>(
            s->fbuf[F_EZ][c->parity], s->fbuf[F_HX][c->parity], s->fbuf[F_HY][c->parity], s->pitch, s->dsg_i0,
            s->dsg_j0, W, H, out);
        c->launches++;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string("edge-weight record: ") + cudaGetErrorString(e);
        return FDTD_ECUDA;
    }
    return FDTD_OK;
}

int adj_next_boundary(const fdtd_ctx* c, int64_t t) {
    const AdjState* A = (const AdjState*)c->adj;
    if (!A || A->every <= 0) return 1 << 30;
    return (int)(A->every - t % A->every);
}

void adj_free(fdtd_ctx* c) {
    AdjState* A = (AdjState*)c->adj;
    if (!A) return;
    cudaStreamSynchronize(c->stream);
    for (float* p : A->ckpt)
        if (p) cudaFree(p);
    for (float* p : A->hist)
        if (p) cudaFree(p);
    delete A;
    c->adj = nullptr;
    c->dirty = true;   // descriptors drop the recording pointers
}

}  // namespace gem

using namespace gem;

extern "C" {

int fdtd_set_checkpointing(fdtd_ctx* c, int every) {
    if (!c) return FDTD_EINVAL;
    if (c->dims != 2) {
        c->err = "checkpointed reverse mode is 2D only";
        return FDTD_EINVAL;
    }
    for (const Scene2* s : c->s2)
        if (s->split) {
            c->err = "reverse mode covers the CPML and PEC boundaries, not the split-field PML";
            return FDTD_EINVAL;
        }
    if (ctx_has_slab(c)) {
        c->err = "reverse mode covers whole grids, not slab sub-domains";
        return FDTD_EINVAL;
    }
    if (every < 0) {
        c->err = "checkpoint interval must be >= 0";
        return FDTD_EINVAL;
    }
    adj_free(c);
    if (every > 0) {
        AdjState* A = new AdjState();
        A->every = every;
        A->store = c->opt_adj_store != 0;
        A->edges = c->opt_adj_store == 2;
        c->adj = A;
    }
    return FDTD_OK;
}

// the reverse sweep shared by fdtd_adjoint_grad (edges = 0: dL/deps_r) and
// fdtd_edge_grad (edges = 1: dL/dw of the 11 edge classes)
static int reverse_run(fdtd_ctx* c, const float* dLdF_re, const float* dLdF_im, float* grad, int on_device,
                       int edges) {
    if (!c || !dLdF_re || !dLdF_im || !grad) return FDTD_EINVAL;
    AdjState* A = (AdjState*)c->adj;
    if (c->dims != 2 || !A || A->every <= 0) {
        c->err = "reverse mode needs a 2D forward run with checkpointing enabled";
        return FDTD_ESTATE;
    }
    if (A->edges != edges) {
        c->err = edges ? "fdtd_edge_grad needs a forward run recorded with FDTD_OPT_ADJ_STORE = 2"
                       : "this forward run was recorded for edge-weight gradients (FDTD_OPT_ADJ_STORE = 2): "
                         "call fdtd_edge_grad";
        return FDTD_ESTATE;
    }
    const int planes = edges ? 3 : 1, n_out = edges ? FDTD_EDGE_CLASSES : 1;
    const int64_t N = c->t;
    const int ns = (int)c->s2.size();
    const int64_t nseg = N >= 1 ? (N - 1) / A->every + 1 : 0;
    for (Scene2* s : c->s2)
        if (!s->d_dsg) {
            c->err = "every scene needs a design rectangle (fdtd_set_design)";
            return FDTD_ESTATE;
        }
    {
        const std::vector<float*>& have = A->store ? A->hist : A->ckpt;
        bool ok = N >= 1 && (int64_t)have.size() >= nseg * ns;
        for (int64_t q = 0; ok && q < nseg * ns; q++) ok = have[(size_t)q] != nullptr;
        if (!ok) {
            c->err = "no recorded forward run to reverse";
            return FDTD_ESTATE;
        }
    }
    cudaStream_t st = c->stream;
    auto cuda_err = [&](cudaError_t e, const char* what) {
        c->err = std::string(what) + ": " + cudaGetErrorString(e);
        return FDTD_ECUDA;
    };
    // per scene: adjoint source table over all cell monitors of that scene
    std::vector<std::vector<Sample2>> srcs(ns);
    std::vector<std::vector<float>> tab(ns);
    std::vector<int> n_adj(ns, 0);
    {
        size_t off = 0;
        for (const DftMon& m : c->mons) {
            if (m.plane_k >= 0) continue;
            n_adj[m.scene] += m.n_cells;
        }
        for (int k = 0; k < ns; k++) tab[k].assign((size_t)N * std::max(1, n_adj[k]), 0.f);
        std::vector<int> used(ns, 0);
        for (const DftMon& m : c->mons) {
            if (m.plane_k >= 0) continue;
            const Scene2* s = c->s2[m.scene];
            for (int q = 0; q < m.n_cells; q++) {
                const Sample2 cell = s->samples[m.slot0 + q];
                Sample2 sp;
                sp.i = cell.i; sp.j = cell.j; sp.comp = 0; sp.slot = used[m.scene] + q;
                srcs[m.scene].push_back(sp);
                for (int64_t n = 0; n < N; n++) {
                    double g = 0.0;
                    for (int f = 0; f < m.n_freq; f++) {
                        const size_t id = off + (size_t)q * m.n_freq + f;
                        double ph = m.freqs[f] * s->dt * (double)(n + 1);
                        ph -= floor(ph);
                        g += ((double)dLdF_re[id] * cos(2.0 * M_PI * ph) - (double)dLdF_im[id] * sin(2.0 * M_PI * ph)) * s->dt;
                    }
                    tab[m.scene][(size_t)n * n_adj[m.scene] + sp.slot] = (float)g;
                }
            }
            used[m.scene] += m.n_cells;
            off += (size_t)m.n_cells * m.n_freq;
        }
    }
    // device buffers: adjoint state (ping-pong), recording, gradient, dC/deps, source tables
    const int every = A->every;
    std::vector<float*> abuf;   // [scene][F_COUNT2][2]
    std::vector<void*> to_free;
    auto dmalloc = [&](size_t bytes, void** p) {
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        to_free.push_back(*p);
        return true;
    };
    auto cleanup = [&]() {
        cudaStreamSynchronize(st);
        for (void* p : to_free) cudaFree(p);
    };
    std::vector<TmzDev> fwd(ns), adj(ns);
    std::vector<Task> tasks, tasks_g, tasks_l, tasks_gd, tasks_n;   // interior, CPML, lite, CPML + design, narrow
    std::vector<Sample2> tsrc;
    std::vector<float*> rec_of(ns), erec_of(ns), grad_of(ns), fac_of(ns);
    const int T = c->opt_tblock, seg = c->opt_segment, warps = c->opt_warps, gwarps = 2, lwarps = 4;
    for (int k = 0; k < ns; k++) {
        Scene2* s = c->s2[k];
        const size_t fb = field_bytes(s), hw = design_cells(s);
        float *aset = nullptr, *rec = nullptr, *erec = nullptr, *gr = nullptr, *src = nullptr, *fac = nullptr;
        if (!dmalloc(F_COUNT2 * 2 * fb, (void**)&aset) ||
            (!A->store && !dmalloc((size_t)every * hw * sizeof(float), (void**)&rec)) ||
            !dmalloc((size_t)every * planes * hw * sizeof(float), (void**)&erec) ||
            !dmalloc(n_out * hw * sizeof(float), (void**)&gr) || !dmalloc(hw * sizeof(float), (void**)&fac) ||
            !dmalloc(tab[k].size() * sizeof(float), (void**)&src)) {
            cleanup();
            c->err = "adjoint: out of device memory";
            return FDTD_ENOMEM;
        }
        cudaMemsetAsync(aset, 0, F_COUNT2 * 2 * fb, st);
        cudaMemsetAsync(gr, 0, n_out * hw * sizeof(float), st);
        cudaMemcpyAsync(src, tab[k].data(), tab[k].size() * sizeof(float), cudaMemcpyHostToDevice, st);
        // eq. (7) with D = eps0 eps_r + sigma dt / 2: Ca = (eps0 eps_r - sigma dt / 2) / D,
        // Cb = dt / D, so dCb/deps_r = -eps0 dt / D^2 = (-eps0 / D) Cb and
        // dCa/deps_r = eps0 sigma dt / D^2 = -sigma dCb/deps_r; the per-cell factor
        // of sum_n e^{n+1} r^n is -eps0 / D, formed when the design was set
        cudaMemcpyAsync(fac, s->d_dsg_fac, hw * sizeof(float), cudaMemcpyDeviceToDevice, st);
        for (int f = 0; f < F_COUNT2; f++)
            for (int p = 0; p < 2; p++) abuf.push_back((float*)((char*)aset + (f * 2 + p) * fb));
        // forward descriptor for the recompute, adjoint descriptor for the reverse sweep
        TmzDev d;
        cudaError_t e = cudaMemcpy(&d, c->d_scenes + k, sizeof(TmzDev), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_err(e, "adjoint: read descriptor");
        }
        d.dsg_rec = rec;
        d.dsg_rec_len = every;
        d.grad = gr;
        d.adj_rec = erec;
        d.adj_src = src;
        d.n_adj = std::max(1, n_adj[k]);
        fwd[k] = d;
        rec_of[k] = rec;
        erec_of[k] = erec;
        grad_of[k] = gr;
        fac_of[k] = fac;
        TmzDev a = d;
        for (int f = 0; f < F_COUNT2; f++)
            for (int p = 0; p < 2; p++) a.f[f][p] = abuf[(size_t)k * F_COUNT2 * 2 + f * 2 + p];
        a.rec = nullptr;
        a.n_rec = 0;
        a.adj_edges = edges;
        adj[k] = a;
        // adjoint tasks: general if a CPML slab, the design rectangle or an
        // adjoint source is within reach, or the strip is ragged.  As in the
        // forward, the columns holding the CPML x-slabs go to narrow lane-group
        // tasks when the layer is shallow enough and the design clear of them,
        // the strips between them carrying a column limit, and the row segments
        // start and end at the y-slab's reach.
        const int wout = STRIP - 2 * HALO;
        const size_t first = tasks.size(), first_g = tasks_g.size(), first_l = tasks_l.size(),
                     first_gd = tasks_gd.size(), first_n = tasks_n.size();
        const int segg = c->opt_segment_b > 0 ? c->opt_segment_b : std::max(8, seg / 2);
        const int xr = (s->nx - NG_OWN + 3) / 4 * 4;
        const bool nar = s->npml > 0 && s->nx >= 2 * NG_OWN + 8 && NG_OWN - HALO >= s->npml &&
                         xr <= s->nx - s->npml - MAX_TB &&
                         !(s->dsg_i0 < NG_OWN + HALO || s->dsg_i0 + s->dsg_w > xr - HALO);
        auto owned_end = [&](int x0) { return nar ? std::min(x0 + wout, xr) : x0 + wout; };
        auto add_srcs = [&](Task& t, int lx0, int lx1, int ly0, int ly1) {
            t.samp_begin = (int)tsrc.size();
            for (const Sample2& sp : srcs[k])
                if (sp.i >= lx0 && sp.i < lx1 && sp.j >= ly0 && sp.j < ly1) tsrc.push_back(sp);
            t.samp_end = (int)tsrc.size();
        };
        if (nar) {
            for (int side = 0; side < 2; side++) {
                const int x0 = side == 0 ? 0 : xr, xe = side == 0 ? NG_OWN : s->nx;
                for (int y = 0; y < s->ny; y += segg) {
                    Task t;
                    t.scene = k; t.x0 = x0; t.ya = y; t.yb = std::min(y + segg, s->ny); t.flags = TASK_PML; t.xe = xe;
                    add_srcs(t, x0 - HALO, x0 - HALO + 4 * NG_LANES, t.ya - MAX_TB, t.yb + MAX_TB);
                    tasks_n.push_back(t);
                }
            }
            const int per_warp = 32 / NG_LANES;
            while ((tasks_n.size() - first_n) % per_warp) {
                Task t = tasks_n[first_n + (tasks_n.size() - first_n) / per_warp * per_warp];
                t.flags |= TASK_NOSTORE;
                tasks_n.push_back(t);
            }
        }
        std::vector<std::pair<int, int>> segs;
        {
            const int y_lo = s->npml > 0 ? std::min(s->ny, s->npml + MAX_TB) : 0;
            const int y_hi = s->npml > 0 ? std::max(y_lo, s->ny - s->npml - MAX_TB) : s->ny;
            for (int y = 0; y < y_lo; y += segg) segs.emplace_back(y, std::min(y + segg, y_lo));
            for (int y = y_lo; y < y_hi; y += seg) segs.emplace_back(y, std::min(y + seg, y_hi));
            for (int y = y_hi; y < s->ny; y += segg) segs.emplace_back(y, std::min(y + segg, s->ny));
        }
        for (const auto& sgm : segs) {
            const int ya = sgm.first;
            for (int x0 = nar ? NG_OWN : 0; x0 < (nar ? xr : s->nx); x0 += wout) {
                const int lx0 = x0 - HALO, lx1 = x0 - HALO + STRIP;
                auto make = [&](int y0, int y1, bool* gen) {
                    Task t;
                    t.scene = k; t.x0 = x0; t.ya = y0; t.yb = y1; t.flags = 0; t.xe = nar ? owned_end(x0) : 0;
                    const int ly0 = y0 - MAX_TB, ly1 = y1 + MAX_TB;
                    const bool xslab = !nar && (lx0 < s->npml || lx1 > s->nx - s->npml);
                    if (s->npml > 0 && (xslab || ly0 < s->npml || ly1 > s->ny - s->npml))
                        t.flags |= TASK_PML;
                    if (s->dsg_i0 < lx1 && s->dsg_i0 + s->dsg_w > lx0 && s->dsg_j0 < ly1 && s->dsg_j0 + s->dsg_h > ly0)
                        t.flags |= TASK_DSG;
                    add_srcs(t, lx0, lx1, ly0, ly1);
                    *gen = t.flags != 0 || t.samp_end > t.samp_begin || (!nar && x0 + wout > s->nx);
                    return t;
                };
                const int yb = sgm.second;
                bool gen;
                const size_t mark = tsrc.size();
                Task t = make(ya, yb, &gen);
                if (!gen) {
                    tasks.push_back(t);
                } else {
                    tsrc.resize(mark);
                    for (int y = ya; y < yb; y += segg) {
                        bool g2;
                        Task t2 = make(y, std::min(y + segg, yb), &g2);
                        (t2.flags & TASK_PML ? (t2.flags & TASK_DSG ? tasks_gd : tasks_g) : tasks_l).push_back(t2);
                    }
                }
            }
        }
        Task pad;
        memset(&pad, 0, sizeof(pad));
        pad.scene = -1;
        if (tasks.size() > first)
            while ((tasks.size() - first) % warps) tasks.push_back(pad);
        if (tasks_g.size() > first_g)
            while ((tasks_g.size() - first_g) % gwarps) tasks_g.push_back(pad);
        if (tasks_l.size() > first_l)
            while ((tasks_l.size() - first_l) % lwarps) tasks_l.push_back(pad);
        if (tasks_gd.size() > first_gd)
            while ((tasks_gd.size() - first_gd) % gwarps) tasks_gd.push_back(pad);
        if (tasks_n.size() > first_n)   // whole CTAs of gwarps warps; a padding warp returns
            while ((tasks_n.size() - first_n) % (gwarps * 32 / NG_LANES)) tasks_n.push_back(pad);
    }
    TmzDev *d_fwd = nullptr, *d_adj = nullptr;
    Task *d_t = nullptr, *d_tg = nullptr, *d_tl = nullptr, *d_tgd = nullptr, *d_tn = nullptr;
    Sample2* d_src = nullptr;
    if (!dmalloc(ns * sizeof(TmzDev), (void**)&d_fwd) || !dmalloc(ns * sizeof(TmzDev), (void**)&d_adj) ||
        !dmalloc(tasks.size() * sizeof(Task), (void**)&d_t) || !dmalloc(tasks_g.size() * sizeof(Task), (void**)&d_tg) ||
        !dmalloc(tasks_l.size() * sizeof(Task), (void**)&d_tl) || !dmalloc(tasks_gd.size() * sizeof(Task), (void**)&d_tgd) ||
        !dmalloc(tasks_n.size() * sizeof(Task), (void**)&d_tn) ||
        !dmalloc(tsrc.size() * sizeof(Sample2), (void**)&d_src)) {
        cleanup();
        c->err = "adjoint: out of device memory";
        return FDTD_ENOMEM;
    }
    cudaMemcpyAsync(d_adj, adj.data(), ns * sizeof(TmzDev), cudaMemcpyHostToDevice, st);
    if (!tasks.empty()) cudaMemcpyAsync(d_t, tasks.data(), tasks.size() * sizeof(Task), cudaMemcpyHostToDevice, st);
    if (!tasks_g.empty()) cudaMemcpyAsync(d_tg, tasks_g.data(), tasks_g.size() * sizeof(Task), cudaMemcpyHostToDevice, st);
    if (!tasks_l.empty()) cudaMemcpyAsync(d_tl, tasks_l.data(), tasks_l.size() * sizeof(Task), cudaMemcpyHostToDevice, st);
    if (!tasks_gd.empty())
        cudaMemcpyAsync(d_tgd, tasks_gd.data(), tasks_gd.size() * sizeof(Task), cudaMemcpyHostToDevice, st);
    if (!tasks_n.empty()) cudaMemcpyAsync(d_tn, tasks_n.data(), tasks_n.size() * sizeof(Task), cudaMemcpyHostToDevice, st);
    if (!tsrc.empty()) cudaMemcpyAsync(d_src, tsrc.data(), tsrc.size() * sizeof(Sample2), cudaMemcpyHostToDevice, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_err(e, "adjoint: upload");
    }

    // checkpoint mode: swap the forward descriptors in for the recompute (recording on)
    TmzDev* saved_scenes = c->d_scenes;
    if (!A->store) c->d_scenes = d_fwd;
    int apar = 0;
    int rc = FDTD_OK;
    for (int64_t sg = nseg - 1; sg >= 0 && rc == FDTD_OK; sg--) {
        const int64_t a0 = sg * every, len = std::min<int64_t>(every, N - a0);
        for (int k = 0; k < ns; k++) {
            fwd[k].dsg_rec_n0 = a0;
            adj[k].dsg_rec_n0 = a0;
        }
        // the adjoint descriptors see this segment's base step
        cudaMemcpyAsync(d_adj, adj.data(), ns * sizeof(TmzDev), cudaMemcpyHostToDevice, st);
        if (!A->store) {
            // restore the checkpoint into buffer 0 and recompute the segment, recording r^n
            for (int k = 0; k < ns && rc == FDTD_OK; k++) {
                Scene2* s = c->s2[k];
                const size_t fb = field_bytes(s);
                const float* p = A->ckpt[(size_t)sg * ns + k];
                for (int f = 0; f < F_COUNT2; f++) {
                    e = cudaMemcpyAsync(s->fbuf[f][0], (const char*)p + f * fb, fb, cudaMemcpyDeviceToDevice, st);
                    if (e != cudaSuccess) rc = cuda_err(e, "adjoint: restore");
                }
            }
            if (rc) break;
            cudaMemcpyAsync(d_fwd, fwd.data(), ns * sizeof(TmzDev), cudaMemcpyHostToDevice, st);
            c->parity = 0;
            for (int64_t q = 0; q < len && rc == FDTD_OK;) {
                const int done = (int)std::min<int64_t>(T, len - q);
                rc = tmz_fused_launch(c, done, warps, a0 + q, c->parity);
                c->parity ^= 1;
                q += done;
            }
            if (rc) break;
        }
        // reverse the segment, T reverse steps per launch; the CPML and lite
        // variants run on their own streams beside the interior one
        AdjLists L;
        L.t0 = d_t; L.n0 = (int)tasks.size(); L.w0 = warps;
        L.sq = 1;
        for (const Scene2* s : c->s2) L.sq = L.sq && s->dx == s->dy;
        L.t1 = d_tg; L.n1 = (int)tasks_g.size(); L.w1 = gwarps;
        L.t2 = d_tl; L.n2 = (int)tasks_l.size(); L.w2 = lwarps;
        L.t3 = d_tgd; L.n3 = (int)tasks_gd.size();
        L.tn = d_tn; L.nn = (int)tasks_n.size();
        const bool fork1 = L.n1 > 0 || L.n3 > 0 || L.nn > 0, fork2 = L.n2 > 0;
        for (int64_t q = len; q > 0 && rc == FDTD_OK;) {
            const int done = (int)std::min<int64_t>(T, q);
            const long long n_top = a0 + q - 1;
            if (fork1 || fork2) {
                cudaEventRecord(c->ev_fork, st);
                if (fork1) cudaStreamWaitEvent(c->aux, c->ev_fork, 0);
                if (fork2) cudaStreamWaitEvent(c->aux2, c->ev_fork, 0);
            }
            cudaStream_t s1 = fork1 ? c->aux : st, s2 = fork2 ? c->aux2 : st;
            switch (done) {
                case 1: e = launch_adj_T<1>(d_adj, L, d_src, apar, n_top, st, s1, s2); break;
                case 2: e = launch_adj_T<2>(d_adj, L, d_src, apar, n_top, st, s1, s2); break;
                case 3: e = launch_adj_T<3>(d_adj, L, d_src, apar, n_top, st, s1, s2); break;
                default: e = launch_adj_T<4>(d_adj, L, d_src, apar, n_top, st, s1, s2); break;
            }
            c->launches += (L.n0 > 0) + (L.n1 > 0) + (L.n2 > 0) + (L.n3 > 0);
            if (fork1) {
                cudaEventRecord(c->ev_join, c->aux);
                cudaStreamWaitEvent(st, c->ev_join, 0);
            }
            if (fork2) {
                cudaEventRecord(c->ev_join2, c->aux2);
                cudaStreamWaitEvent(st, c->ev_join2, 0);
            }
            if (e != cudaSuccess) rc = cuda_err(e, "adjoint launch");
            apar ^= 1;
            q -= done;
        }
        if (rc) break;
        // fold the segment's e and recorded r^n into dL/deps_r
        for (int k = 0; k < ns; k++) {
            const Scene2* s = c->s2[k];
            const int hw = (int)design_cells(s);
            if (edges) {
                const float* prev = sg > 0 ? A->hist[(size_t)(sg - 1) * ns + k] + (size_t)(every - 1) * 3 * window_cells(s)
                                           : nullptr;
                k_edge_reduce<<<(hw + 127) / 128, 128, 0, st>>>(A->hist[(size_t)sg * ns + k], prev, erec_of[k],
                                                                grad_of[k], s->dsg_w, s->dsg_h, (int)len);
            } else {
                const float* r = A->store ? A->hist[(size_t)sg * ns + k] : rec_of[k];
                k_grad_reduce<<<(hw + 255) / 256, 256, 0, st>>>(r, erec_of[k], fac_of[k], grad_of[k], hw, (int)len);
            }
            c->launches++;
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_err(e, "adjoint: gradient reduction");
    }
    c->d_scenes = saved_scenes;
    if (rc == FDTD_OK) {
        size_t off = 0;
        for (int k = 0; k < ns; k++) {
            const size_t hw = (size_t)n_out * c->s2[k]->dsg_w * c->s2[k]->dsg_h;
            e = cudaMemcpyAsync(grad + off, adj[k].grad, hw * sizeof(float),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) {
                rc = cuda_err(e, "adjoint: gradient copy");
                break;
            }
            off += hw;
        }
    }
    cleanup();
    return rc;
}

int fdtd_adjoint_grad(fdtd_ctx* c, const float* dLdF_re, const float* dLdF_im, float* grad, int on_device) {
    NvtxRange nvtx("fdtd_adjoint_grad");
    return reverse_run(c, dLdF_re, dLdF_im, grad, on_device, 0);
}

int fdtd_edge_grad(fdtd_ctx* c, const float* dLdF_re, const float* dLdF_im, float* grad, int on_device) {
    NvtxRange nvtx("fdtd_edge_grad");
    return reverse_run(c, dLdF_re, dLdF_im, grad, on_device, 1);
}

}  // extern "C"

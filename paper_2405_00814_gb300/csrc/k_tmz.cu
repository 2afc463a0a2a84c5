// 2D TMz kernels for sm_103a.
//
// The leapfrog step of Sec. III-B (eqs. (7)-(9), rotated to TMz) is the two
// message-passing layers of Prop. 2 with the graph kept implicit in the grid:
//   layer 1:  Hx -= Db_y (dEz/dy + psi_Hxy),  Hy += Db_x (dEz/dx + psi_Hyx)
//   layer 2:  Ez  = Ca Ez + Cb/dx (dHy + psi_Ezx) - Cb/dy (dHx + psi_Ezy)
// with CPML auxiliaries psi = b psi + c dF inside the absorbing slabs.
//
// k_tmz_fused -- the hot path.  One warp streams a 128-column strip (4 columns
// per lane, float4 loads) up a segment of rows.  Each row enters through a
// cp.async pipeline into lane-private shared-memory stages, then lives in a
// register ring while T time levels are applied to it in a skewed wavefront:
// at row r, level t updates row r - t (H then E), so a row leaves the ring
// T steps newer than it came in.  x-neighbours come from warp shuffles (the
// right Ez for layer 1, the left Hy for layer 2); y-neighbours are the adjacent
// ring slots.  The strip's outer lane on each side is a halo whose values go
// stale by one column per level, so T <= 4 keeps the 120 inner columns exact.
// Each launch reads buffer `parity` and writes 1 - parity.  HBM traffic per
// cell and launch is the 12 B of fields + 1 B of material read and 12 B written
// (plus halo re-reads), for T steps: the single-sweep 25 B per cell-update is
// divided by T.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "gem_internal.h"

namespace gem {

// Three task kinds.  CPML tasks (general_task<T, true>) stage 7 float4 slots per
// lane per row -- Ez Hx Hy and psi_Ezx psi_Ezy psi_Hxy psi_Hyx -- plus the row's
// four y-profile scalars, and keep PF_B rows in flight.  Lite tasks (design
// rectangle, source, probes, ragged edge; general_task<T, false>) stage Ez Hx Hy
// and, inside the design band, the row's Ca, Cb/dx, Cb/dy, so that no level of
// the wavefront waits on a global load.  Interior tasks (k_tmz_interior) stage
// only Ez Hx Hy, with a register cap that lets four warps share each SM
// sub-partition.  Lite and interior warps hold Q_I = 8 stages (a power of two,
// so the stage of a row is a mask) with 8 - T rows in flight.
constexpr int PF_B = 3;
constexpr int Q_I = 8;
__host__ __device__ constexpr int nslot_of(bool pml) { return pml ? 7 : 3; }
__host__ __device__ constexpr int stage_f4(bool pml) { return nslot_of(pml) * 32 + 8; }   // + 32 uint32 material words
__host__ __device__ constexpr int stages_for(int T, bool pml) { return pml ? T + PF_B : Q_I; }
__host__ __device__ constexpr int pf_of(int T, bool pml) { return pml ? PF_B : Q_I - T; }
// general tasks: CPML kind adds one float4 of y-profile scalars after the
// material words; lite kind has three design-coefficient slots after the fields
__host__ __device__ constexpr int gen_nslot(bool pml) { return pml ? 7 : 6; }
__host__ __device__ constexpr int gen_stage_f4(bool pml, int groups = 1) {
    return gen_nslot(pml) * 32 + 8 + (pml ? groups : 0);
}

// V: 0 interior, 1 CPML, 2 lite, 3 split-field layer; 5, 6: CPML, lite keeping
// the design window (edge-weight reverse mode); 7: CPML without design code;
// 8: CPML without design code in narrow lane groups (NG_LANES lanes per task)
size_t tmz_fused_smem(int T, int warps, int V) {
    if (V == 0) return (size_t)warps * stages_for(T, false) * stage_f4(false) * sizeof(float4);
    if (V == 8) return (size_t)warps * stages_for(T, true) * gen_stage_f4(true, 32 / NG_LANES) * sizeof(float4);
    const bool pml = V == 1 || V == 3 || V == 5 || V == 7;   // 3 split layer, 5 window-keeping, 7 design-free CPML
    return (size_t)warps * stages_for(T, pml) * gen_stage_f4(pml) * sizeof(float4);
}

__device__ __forceinline__ size_t sidx(int pitch, int i, int j) {
    return (size_t)(j + PAD_Y) * (size_t)pitch + (size_t)(i + PAD_X);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool pred) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    int n = pred ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ float comp4(const float4& v, int c) {
    return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

__device__ __forceinline__ void add4(float4& v, int c, float a) {
    if (c == 0) v.x += a;
    else if (c == 1) v.y += a;
    else if (c == 2) v.z += a;
    else v.w += a;
}

// Ez = Ca Ez + Cb/dx (dhy + psi_x) - Cb/dy (dhx + psi_y)
__device__ __forceinline__ float e_upd(float e, float dhy, float dhx, const float4& co) {
    return co.x * e + co.y * dhy - co.z * dhx;
}
// square cells (dx = dy, so Cb/dx = Cb/dy): co = (Ca, Cb/dx), one product for
// the curl
__device__ __forceinline__ float e_upd(float e, float dhy, float dhx, const float2& co) {
    return co.x * e + co.y * (dhy - dhx);
}

struct Prof {
    const float* p;
    int pitch, rows;
    __device__ __forceinline__ float bEx(int cs) const { return p[cs]; }
    __device__ __forceinline__ float cEx(int cs) const { return p[pitch + cs]; }
    __device__ __forceinline__ float bHx(int cs) const { return p[2 * pitch + cs]; }
    __device__ __forceinline__ float cHx(int cs) const { return p[3 * pitch + cs]; }
    __device__ __forceinline__ float bEy(int rs) const { return p[4 * pitch + rs]; }
    __device__ __forceinline__ float cEy(int rs) const { return p[4 * pitch + rows + rs]; }
    __device__ __forceinline__ float bHy(int rs) const { return p[4 * pitch + 2 * rows + rs]; }
    __device__ __forceinline__ float cHy(int rs) const { return p[4 * pitch + 3 * rows + rs]; }
};

// ===========================================================================
// fused, temporally blocked kernel
// ===========================================================================
// One warp's task of the general kernel (any task: CPML slab, design rectangle,
// source, probes, ragged edge).  coef_s is the scene's coefficient table (shared
// or global memory); stage0 the warp's Q x STAGE_F4 float4 staging area.
//
// G < 32: the warp runs 32 / G independent tasks, one per group of G lanes (a
// narrow strip of (G - 2) * 4 owned columns each, e.g. the columns of an x-slab
// of the CPML): x-neighbours come from width-G shuffles, every group streams as
// many rows as the longest task of the warp (a shorter one re-reads its last
// row and stores nothing past it), and the source and the samples are read
// from memory, not shuffled, since the groups' rows differ.
template <int T, bool PML, bool SPL = false, bool WREC = false, bool DSG = true, int G = 32>
__device__ __forceinline__ void general_task(const TmzDev* __restrict__ S, const Task& tk,
                                             const Sample2* __restrict__ samps, int parity, long long n0,
                                             const float4* coef_s, float4* stage0, int lane) {
    static_assert(G == 32 || (G >= 4 && G < 32 && (G & (G - 1)) == 0), "lane groups of 4, 8 or 16 lanes");
    constexpr int PF = pf_of(T, PML);
    constexpr int NSLOT = gen_nslot(PML);
    constexpr int STAGE_F4 = gen_stage_f4(PML, 32 / G);
    constexpr int Q = stages_for(T, PML);
    constexpr bool SD = !PML;   // design coefficients come staged (lite kind)
    const int pitch = S->pitch, nx = S->nx, ny = S->ny;
    const float* __restrict__ ez_in = S->f[F_EZ][parity];
    const float* __restrict__ hx_in = S->f[F_HX][parity];
    const float* __restrict__ hy_in = S->f[F_HY][parity];
    float* __restrict__ ez_out = S->f[F_EZ][parity ^ 1];
    float* __restrict__ hx_out = S->f[F_HX][parity ^ 1];
    float* __restrict__ hy_out = S->f[F_HY][parity ^ 1];
    const uint8_t* __restrict__ mat = S->mat;
    const float dbx = S->dbx, dby = S->dby;

    const int gl = lane & (G - 1);             // lane within the task's group
    const int grp = lane / G;                  // the group (0 for whole-warp tasks)
    const int cx = tk.x0 - HALO + 4 * gl;      // first of this lane's 4 columns
    const int cs = cx + PAD_X;                 // its storage column (>= 4)
    // owned: not a halo lane, inside the grid and before the task's column limit
    const bool out_lane = (gl >= HALO / 4) && (gl < G - HALO / 4) && (cx < nx) && (tk.xe == 0 || cx < tk.xe) &&
                          !(tk.flags & TASK_NOSTORE);
    const int s_row = tk.ya - T;               // first row streamed
    const int r_last = tk.yb + T - 1;          // last row streamed
    // iterations of the row loop: the longest stream of the warp's tasks
    int n_iter = r_last - s_row + 1;
    if constexpr (G < 32) n_iter = (int)__reduce_max_sync(0xffffffffu, (unsigned)n_iter);

    // CPML: lanes whose columns touch an x-slab carry psi_Ezx / psi_Hyx
    const bool pml = PML && (tk.flags & TASK_PML) != 0;
    const int npml = S->has_pml;
    const int ylo = S->pml_ylo, yhi = S->pml_yhi;   // rows outside [ylo, yhi) may lie in a y-slab
    const Prof pr{S->prof, pitch, S->rows};
    bool lane_px = false;
    float4 bex4 = make_float4(0, 0, 0, 0), cex4 = bex4, bhx4 = bex4, chx4 = bex4;
    // split-field layer (SPL): depth nsp; the profiles hold Ca, Cb/d of E and
    // Da, Db/d of H per axis, and the stage's psi_Ezy slot carries Ezy
    const int nsp = SPL ? S->split : 0;
    const bool lane_sx = SPL && pml && ((cx < nsp) || (cx + 3 >= nx - nsp));
    if (lane_sx) {
        bex4 = make_float4(pr.bEx(cs), pr.bEx(cs + 1), pr.bEx(cs + 2), pr.bEx(cs + 3));
        cex4 = make_float4(pr.cEx(cs), pr.cEx(cs + 1), pr.cEx(cs + 2), pr.cEx(cs + 3));
        bhx4 = make_float4(pr.bHx(cs), pr.bHx(cs + 1), pr.bHx(cs + 2), pr.bHx(cs + 3));
        chx4 = make_float4(pr.cHx(cs), pr.cHx(cs + 1), pr.cHx(cs + 2), pr.cHx(cs + 3));
    }
    auto srow = [&](int row) { return (row < nsp) || (row >= ny - nsp); };   // a split-layer row (E or H)
    if (!SPL && pml) {
        lane_px = (cx < npml) || (cx + 3 >= nx - npml);
        if (lane_px) {
            bex4 = make_float4(pr.bEx(cs), pr.bEx(cs + 1), pr.bEx(cs + 2), pr.bEx(cs + 3));
            cex4 = make_float4(pr.cEx(cs), pr.cEx(cs + 1), pr.cEx(cs + 2), pr.cEx(cs + 3));
            bhx4 = make_float4(pr.bHx(cs), pr.bHx(cs + 1), pr.bHx(cs + 2), pr.bHx(cs + 3));
            chx4 = make_float4(pr.cHx(cs), pr.cHx(cs + 1), pr.cHx(cs + 2), pr.cHx(cs + 3));
        }
    }
    float* psi_in[4] = {S->f[F_PEZX][parity], S->f[F_PEZY][parity], S->f[F_PHXY][parity],
                        S->f[F_PHYX][parity]};
    float* psi_out[4] = {S->f[F_PEZX][parity ^ 1], S->f[F_PEZY][parity ^ 1],
                         S->f[F_PHXY][parity ^ 1], S->f[F_PHYX][parity ^ 1]};

    // design rectangle (continuous permittivity); scene scalars live in registers
    const bool dsg = DSG && (tk.flags & TASK_DSG) != 0;   // DSG = false: compiled without design code
    const int dsg_i0 = S->dsg_i0, dsg_j0 = S->dsg_j0, dsg_w = S->dsg_w, dsg_h = S->dsg_h;
    const float4* __restrict__ dsg_coef = S->dsg_coef;
    const float* __restrict__ band = S->dsg_band;
    const size_t band_plane = (size_t)dsg_h * pitch;
    float* const dsg_rec = S->dsg_rec;
    const long long rec_n0 = S->dsg_rec_n0, rec_len = S->dsg_rec_len;
    // probes and monitor cells of this task: the first 32 ride in lane registers
    const int n_samp = tk.samp_end - tk.samp_begin;
    const bool has_samp = n_samp > 0;
    Sample2 my_samp;
    my_samp.i = -1; my_samp.j = -1; my_samp.comp = 0; my_samp.slot = 0;
    if (G == 32 && lane < n_samp) my_samp = samps[tk.samp_begin + lane];
    // source: this launch's T waveform values ride in lanes 0..T-1
    const bool has_src = (tk.flags & TASK_SRC) != 0;
    const int src_j = S->src_j, src_j1 = S->src_j1, src_d = S->src_i - cx;
    const long long src_len = S->src_len;
    float wv = 0.f;
    if (G == 32 && has_src && lane < T && n0 + lane < src_len) wv = S->src_wave[n0 + lane];


    // stage the row of iteration i (past its last row, a group re-reads that row)
    auto issue = [&](int i) {
        const int row = G < 32 ? min(s_row + i, r_last) : s_row + i;
        const int q = i % Q;
        float4* st = stage0 + q * STAGE_F4;
        const size_t g = (size_t)(row + PAD_Y) * pitch + cs;
        cp_async16(st + 0 * 32 + lane, ez_in + g, true);
        cp_async16(st + 1 * 32 + lane, hx_in + g, true);
        cp_async16(st + 2 * 32 + lane, hy_in + g, true);
        cp_async4(reinterpret_cast<uint32_t*>(st + NSLOT * 32) + lane, mat + g);
        if constexpr (SD) {
            if (dsg && row >= dsg_j0 && row < dsg_j0 + dsg_h) {
                const float* b = band + (size_t)(row - dsg_j0) * pitch + cs;
                cp_async16(st + 3 * 32 + lane, b, true);
                cp_async16(st + 4 * 32 + lane, b + band_plane, true);
                cp_async16(st + 5 * 32 + lane, b + 2 * band_plane, true);
            }
        }
        if constexpr (SPL) if (pml) {
            // the row's Ca, Cb/dy of E and Da, Db/dy of H, and Ezy
            const bool yrow = srow(row);
            if (yrow && gl < 4)
                cp_async4(reinterpret_cast<float*>(st + NSLOT * 32 + 8 + grp) + gl, pr.p + 4 * pitch + gl * pr.rows + row + PAD_Y);
            if (yrow || lane_sx) cp_async16(st + 4 * 32 + lane, psi_in[1] + g, true);
        }
        if constexpr (PML && !SPL) if (pml) {
            const bool yrow = (row < ylo) || (row >= yhi);
            // the row's bEy, cEy, bHy, cHy
            if (yrow && gl < 4)
                cp_async4(reinterpret_cast<float*>(st + NSLOT * 32 + 8 + grp) + gl, pr.p + 4 * pitch + gl * pr.rows + row + PAD_Y);
            if (lane_px) {
                cp_async16(st + 3 * 32 + lane, psi_in[0] + g, true);
                cp_async16(st + 6 * 32 + lane, psi_in[3] + g, true);
            }
            if (yrow) {
                cp_async16(st + 4 * 32 + lane, psi_in[1] + g, true);
                cp_async16(st + 5 * 32 + lane, psi_in[2] + g, true);
            }
        }
    };

    // register ring: slot k holds row r - k
    float4 E[T + 1], X[T + 2], Y[T + 1];
    uint32_t M[T + 1];
#pragma unroll
    for (int k = 0; k < T + 1; k++) {
        E[k] = make_float4(0, 0, 0, 0);
        Y[k] = E[k];
        M[k] = 0;
    }
#pragma unroll
    for (int k = 0; k < T + 2; k++) X[k] = make_float4(0, 0, 0, 0);

#pragma unroll
    for (int k = 0; k < PF; k++) {
        if (k < n_iter) issue(k);
        cp_commit();
    }

    float* rec = S->rec;
    const int n_rec = S->n_rec;

    // not unrolled: the general body is large, and instruction fetch, not
    // issue, limits these latency-bound warps
#pragma unroll 1
    for (int it = 0; it < n_iter; ++it) {
        const int r = s_row + it;
        cp_wait<PF - 1>();
        // shift the ring and take row r from its stage
#pragma unroll
        for (int k = T + 1; k >= 1; k--) X[k] = X[k - 1];
#pragma unroll
        for (int k = T; k >= 1; k--) {
            E[k] = E[k - 1];
            Y[k] = Y[k - 1];
            M[k] = M[k - 1];
        }
        {
            const float4* st = stage0 + (it % Q) * STAGE_F4;
            E[0] = st[0 * 32 + lane];
            X[0] = st[1 * 32 + lane];
            Y[0] = st[2 * 32 + lane];
            M[0] = reinterpret_cast<const uint32_t*>(st + NSLOT * 32)[lane];
        }

#pragma unroll
        for (int t = 1; t <= T; t++) {
            const int a = r - t;
            if (a < s_row) continue;   // warp-uniform
            float4* sta = stage0 + ((a - s_row) % Q) * STAGE_F4;
            const float* yprof = reinterpret_cast<const float*>(sta + NSLOT * 32 + 8 + grp);
            // ---- layer 1: H at row a from Ez at level t-1 (rows a, a+1) ----
            const float4 e = E[t], eu = E[t - 1];
            const float er = __shfl_down_sync(0xffffffffu, e.x, 1, G);
            float4 dey = make_float4(eu.x - e.x, eu.y - e.y, eu.z - e.z, eu.w - e.w);
            float4 dex = make_float4(e.y - e.x, e.z - e.y, e.w - e.z, er - e.w);
            if constexpr (PML && !SPL) if (pml) {
                if ((a < ylo) || (a >= yhi)) {
                    const float b = yprof[2], c = yprof[3];
                    float4 p = sta[5 * 32 + lane];
                    p.x = b * p.x + c * dey.x;
                    p.y = b * p.y + c * dey.y;
                    p.z = b * p.z + c * dey.z;
                    p.w = b * p.w + c * dey.w;
                    sta[5 * 32 + lane] = p;
                    dey.x += p.x; dey.y += p.y; dey.z += p.z; dey.w += p.w;
                }
                if (lane_px) {
                    float4 p = sta[6 * 32 + lane];
                    p.x = bhx4.x * p.x + chx4.x * dex.x;
                    p.y = bhx4.y * p.y + chx4.y * dex.y;
                    p.z = bhx4.z * p.z + chx4.z * dex.z;
                    p.w = bhx4.w * p.w + chx4.w * dex.w;
                    sta[6 * 32 + lane] = p;
                    dex.x += p.x; dex.y += p.y; dex.z += p.z; dex.w += p.w;
                }
            }
            bool h_done = false;
            if constexpr (SPL) if (pml) {
                // split layer: H damped along the axis its derivative runs along
                // (sigma*), semi-implicit as eq. (7); elsewhere the plain update
                if (srow(a)) {
                    const float da = yprof[2], db = yprof[3];
                    X[t].x = da * X[t].x - db * dey.x; X[t].y = da * X[t].y - db * dey.y;
                    X[t].z = da * X[t].z - db * dey.z; X[t].w = da * X[t].w - db * dey.w;
                } else {
                    X[t].x -= dby * dey.x; X[t].y -= dby * dey.y; X[t].z -= dby * dey.z; X[t].w -= dby * dey.w;
                }
                if (lane_sx) {
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const int i = cx + q;
                        const float hy = comp4(Y[t], q), d = comp4(dex, q);
                        const float v = (i < nsp || i >= nx - nsp) ? comp4(bhx4, q) * hy + comp4(chx4, q) * d : hy + dbx * d;
                        if (q == 0) Y[t].x = v; else if (q == 1) Y[t].y = v; else if (q == 2) Y[t].z = v; else Y[t].w = v;
                    }
                } else {
                    Y[t].x += dbx * dex.x; Y[t].y += dbx * dex.y; Y[t].z += dbx * dex.z; Y[t].w += dbx * dex.w;
                }
                h_done = true;
            }
            if (!h_done) {
                X[t].x -= dby * dey.x; X[t].y -= dby * dey.y; X[t].z -= dby * dey.z; X[t].w -= dby * dey.w;
                Y[t].x += dbx * dex.x; Y[t].y += dbx * dex.y; Y[t].z += dbx * dex.z; Y[t].w += dbx * dex.w;
            }

            // ---- layer 2: Ez at row a from H at level t (rows a, a-1) ----
            const float4 y = Y[t];
            const float yl = __shfl_up_sync(0xffffffffu, y.w, 1, G);
            float4 dhy = make_float4(y.x - yl, y.y - y.x, y.z - y.y, y.w - y.z);
            float4 dhx = make_float4(X[t].x - X[t + 1].x, X[t].y - X[t + 1].y, X[t].z - X[t + 1].z,
                                     X[t].w - X[t + 1].w);
            if constexpr (PML && !SPL) if (pml) {
                if ((a < ylo) || (a >= yhi)) {
                    const float b = yprof[0], c = yprof[1];
                    float4 p = sta[4 * 32 + lane];
                    p.x = b * p.x + c * dhx.x;
                    p.y = b * p.y + c * dhx.y;
                    p.z = b * p.z + c * dhx.z;
                    p.w = b * p.w + c * dhx.w;
                    sta[4 * 32 + lane] = p;
                    dhx.x += p.x; dhx.y += p.y; dhx.z += p.z; dhx.w += p.w;
                }
                if (lane_px) {
                    float4 p = sta[3 * 32 + lane];
                    p.x = bex4.x * p.x + cex4.x * dhy.x;
                    p.y = bex4.y * p.y + cex4.y * dhy.y;
                    p.z = bex4.z * p.z + cex4.z * dhy.z;
                    p.w = bex4.w * p.w + cex4.w * dhy.w;
                    sta[3 * 32 + lane] = p;
                    dhy.x += p.x; dhy.y += p.y; dhy.z += p.z; dhy.w += p.w;
                }
            }
            const uint32_t m = M[t];
            float4 c0 = coef_s[m & 255u], c1 = coef_s[(m >> 8) & 255u];
            float4 c2 = coef_s[(m >> 16) & 255u], c3 = coef_s[m >> 24];
            if (dsg) {
                const int dj = a - dsg_j0;
                if (dj >= 0 && dj < dsg_h) {
                    const int di = cx - dsg_i0;
                    if constexpr (SD) {
                        // the band holds the effective coefficients of every column
                        const float4 ca = sta[3 * 32 + lane], cbx = sta[4 * 32 + lane], cby = sta[5 * 32 + lane];
                        c0 = make_float4(ca.x, cbx.x, cby.x, 0.f);
                        c1 = make_float4(ca.y, cbx.y, cby.y, 0.f);
                        c2 = make_float4(ca.z, cbx.z, cby.z, 0.f);
                        c3 = make_float4(ca.w, cbx.w, cby.w, 0.f);
                    } else {
                        const float4* drow = dsg_coef + (size_t)dj * dsg_w;
                        if (di >= 0 && di < dsg_w) c0 = drow[di];
                        if (di + 1 >= 0 && di + 1 < dsg_w) c1 = drow[di + 1];
                        if (di + 2 >= 0 && di + 2 < dsg_w) c2 = drow[di + 2];
                        if (di + 3 >= 0 && di + 3 < dsg_w) c3 = drow[di + 3];
                    }
                }
            }
            const float4 e_old = E[t];
            E[t].x = e_upd(E[t].x, dhy.x, dhx.x, c0);
            E[t].y = e_upd(E[t].y, dhy.y, dhx.y, c1);
            E[t].z = e_upd(E[t].z, dhy.z, dhx.z, c2);
            E[t].w = e_upd(E[t].w, dhy.w, dhx.w, c3);
            if constexpr (SPL) if (pml) {
                // split layer (Sec. III-C): Ez = Ezx + Ezy with Ezy in the stage,
                // each part advanced with its own axis's coefficients (vacuum cells)
                const bool ly = a < nsp || a > ny - nsp;
                if ((ly || lane_sx) && a >= 1) {
                    float4 zy = sta[4 * 32 + lane];
                    const float4 cq[4] = {c0, c1, c2, c3};
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const int i = cx + q;
                        const bool lx = i < nsp || i > nx - nsp;
                        if (i < 1 || !(lx || ly)) continue;
                        const float ezy0 = comp4(zy, q), ezx0 = comp4(e_old, q) - ezy0;
                        const float ax = lx ? comp4(bex4, q) : cq[q].x, bx = lx ? comp4(cex4, q) : cq[q].y;
                        const float ay = ly ? yprof[0] : cq[q].x, by = ly ? yprof[1] : cq[q].z;
                        const float ezx = ax * ezx0 + bx * comp4(dhy, q);
                        const float ezy = ay * ezy0 - by * comp4(dhx, q);
                        if (q == 0) { zy.x = ezy; E[t].x = ezx + ezy; }
                        else if (q == 1) { zy.y = ezy; E[t].y = ezx + ezy; }
                        else if (q == 2) { zy.z = ezy; E[t].z = ezx + ezy; }
                        else { zy.w = ezy; E[t].w = ezx + ezy; }
                    }
                    sta[4 * 32 + lane] = zy;
                }
            }
            // reverse mode: E^{n+1} - E^n of the owned design cells (before the
            // source), which carries dL/deps_r of step n up to a per-cell factor
            if (!WREC && dsg && dsg_rec) {
                const int dj = a - dsg_j0;
                const long long nr = n0 + (t - 1) - rec_n0;
                if (dj >= 0 && dj < dsg_h && nr >= 0 && nr < rec_len && a >= tk.ya && a < tk.yb && out_lane) {
                    const int di = cx - dsg_i0;
                    float* re = dsg_rec + (size_t)nr * dsg_w * dsg_h + (size_t)dj * dsg_w;
                    const float dv[4] = {E[t].x - e_old.x, E[t].y - e_old.y, E[t].z - e_old.z, E[t].w - e_old.w};
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const int d = di + q;
                        if (d >= 0 && d < dsg_w && cx + q >= tk.x0 && cx + q < tk.x0 + (STRIP - 2 * HALO)) re[d] = dv[q];
                    }
                }
            }

            const long long n = n0 + (t - 1);   // this level makes E^{n+1}
            if (has_src && a >= src_j && a < src_j1) {
                if constexpr (G == 32) {
                    const float w = __shfl_sync(0xffffffffu, wv, t - 1);
                    if (src_d >= 0 && src_d < 4 && n < src_len) add4(E[t], src_d, w);
                } else {
                    if (src_d >= 0 && src_d < 4 && n < src_len) add4(E[t], src_d, S->src_wave[n]);
                }
            }
            // edge-weight gradients: Ez^{n+1} (after the source), Hx^{n+1/2},
            // Hy^{n+1/2} of the owned cells of the window one cell around the design
            if (WREC && dsg && dsg_rec) {
                const int wr = a - (dsg_j0 - 1), W = dsg_w + 2, H = dsg_h + 2;
                const long long nr = n - rec_n0;
                if (wr >= 0 && wr < H && nr >= 0 && nr < rec_len && a >= tk.ya && a < tk.yb && out_lane) {
                    const size_t ww = (size_t)W * H;
                    float* re = dsg_rec + (size_t)nr * 3 * ww + (size_t)wr * W;
                    const int wc = cx - (dsg_i0 - 1);
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const int d = wc + q;
                        if (d >= 0 && d < W && cx + q >= tk.x0 && cx + q < tk.x0 + (STRIP - 2 * HALO)) {
                            re[d] = comp4(E[t], q);
                            re[ww + d] = comp4(X[t], q);
                            re[2 * ww + d] = comp4(Y[t], q);
                        }
                    }
                }
            }
            if (has_samp && a >= tk.ya && a < tk.yb && !(tk.flags & TASK_NOSTORE)) {
                const int nq = G == 32 ? (n_samp < 32 ? n_samp : 32) : 0;   // groups read their samples from memory
                for (int q = 0; q < nq; q++) {
                    if (__shfl_sync(0xffffffffu, my_samp.j, q) != a) continue;   // warp-uniform
                    const int d = __shfl_sync(0xffffffffu, my_samp.i, q) - cx;
                    const int comp = __shfl_sync(0xffffffffu, my_samp.comp, q);
                    const int slot = __shfl_sync(0xffffffffu, my_samp.slot, q);
                    if (d >= 0 && d < 4)
                        rec[n * n_rec + slot] = comp == 0 ? comp4(E[t], d) : (comp == 1 ? comp4(X[t], d) : comp4(Y[t], d));
                }
                for (int q = tk.samp_begin + (G == 32 ? 32 : 0); q < tk.samp_end; q++) {
                    const Sample2 sp = samps[q];
                    const int d = sp.i - cx;
                    if (sp.j == a && d >= 0 && d < 4)
                        rec[n * n_rec + sp.slot] = sp.comp == 0 ? comp4(E[t], d) : (sp.comp == 1 ? comp4(X[t], d) : comp4(Y[t], d));
                }
            }
        }

        // ---- row r - T is T steps newer: write it out ----
        const int o = r - T;
        if (o >= tk.ya && o < tk.yb) {
            const float4* sto = stage0 + ((o - s_row) % Q) * STAGE_F4;
            (void)sto;
            if (out_lane) {
                const size_t g = (size_t)(o + PAD_Y) * pitch + cs;
                if (cx + 3 < nx) {
                    *reinterpret_cast<float4*>(ez_out + g) = E[T];
                    *reinterpret_cast<float4*>(hx_out + g) = X[T];
                    *reinterpret_cast<float4*>(hy_out + g) = Y[T];
                    if constexpr (SPL) if (pml) {
                        if (srow(o) || lane_sx) *reinterpret_cast<float4*>(psi_out[1] + g) = sto[4 * 32 + lane];
                    }
                    if constexpr (PML && !SPL) if (pml) {
                        if ((o < ylo) || (o >= yhi)) {
                            *reinterpret_cast<float4*>(psi_out[1] + g) = sto[4 * 32 + lane];
                            *reinterpret_cast<float4*>(psi_out[2] + g) = sto[5 * 32 + lane];
                        }
                        if (lane_px) {
                            *reinterpret_cast<float4*>(psi_out[0] + g) = sto[3 * 32 + lane];
                            *reinterpret_cast<float4*>(psi_out[3] + g) = sto[6 * 32 + lane];
                        }
                    }
                } else {
                    float4 p0 = make_float4(0, 0, 0, 0), p1 = p0, p2 = p0, p3 = p0;
                    if constexpr (PML) {
                        p0 = sto[3 * 32 + lane]; p1 = sto[4 * 32 + lane];
                        p2 = sto[5 * 32 + lane]; p3 = sto[6 * 32 + lane];
                    }
                    const bool yrow = !SPL && pml && ((o < ylo) || (o >= yhi));
                    const bool srw = SPL && pml && (srow(o) || lane_sx);
                    for (int c = 0; c < 4; c++) {
                        if (cx + c >= nx) break;
                        ez_out[g + c] = comp4(E[T], c);
                        hx_out[g + c] = comp4(X[T], c);
                        hy_out[g + c] = comp4(Y[T], c);
                        if (srw) psi_out[1][g + c] = comp4(p1, c);
                        if (yrow) {
                            psi_out[1][g + c] = comp4(p1, c);
                            psi_out[2][g + c] = comp4(p2, c);
                        }
                        if (pml && lane_px) {
                            psi_out[0][g + c] = comp4(p0, c);
                            psi_out[3][g + c] = comp4(p3, c);
                        }
                    }
                }
            }
        }
        // the stage of row r - T is free: prefetch the row of iteration it + PF into it
        if (it + PF < n_iter) issue(it + PF);
        cp_commit();
    }
    cp_wait<0>();
}

// CPML blocks run 2 warps, lite blocks 4 (the lists are padded to that)
template <int T, bool PML, bool SPL = false, bool WREC = false, bool DSG = true>
__global__ void __launch_bounds__(PML ? 256 : 128, PML ? 1 : 3) k_tmz_fused(const TmzDev* __restrict__ scenes,
                                                   const Task* __restrict__ tasks, int n_tasks,
                                                   const Sample2* __restrict__ samps, int parity,
                                                   long long n0) {
    constexpr int STAGE_F4 = gen_stage_f4(PML);
    constexpr int Q = stages_for(T, PML);
    extern __shared__ float4 smem_f4[];
    __shared__ float4 coef_s[256];

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int warps = blockDim.x >> 5;
    const int tid = blockIdx.x * warps + wib;

    // every block holds tasks of one scene: stage its coefficient table (a
    // block of padding only returns)
    if (tasks[blockIdx.x * warps].scene < 0) return;
    const TmzDev* S = scenes + tasks[blockIdx.x * warps].scene;
    for (int k = threadIdx.x; k < 256; k += blockDim.x) coef_s[k] = S->coef[k];
    __syncthreads();
    if (tid >= n_tasks) return;
    const Task tk = tasks[tid];
    if (tk.scene < 0) return;
    general_task<T, PML, SPL, WREC, DSG>(S, tk, samps, parity, n0, coef_s, smem_f4 + (size_t)wib * Q * STAGE_F4,
                                         lane);
}

// CPML tasks of one T-step block in one launch: the first nw_blocks CTAs run
// whole-warp tasks (y-slab segments, sources, probes; the build without design
// code), the rest run the narrow x-slab tasks, 32 / NG_LANES per warp.  Both
// lists are padded to whole CTAs of one scene.
template <int T>
__global__ void __launch_bounds__(256, 1) k_tmz_cpml_mixed(const TmzDev* __restrict__ scenes,
                                                          const Task* __restrict__ tasks_w, int nw_blocks,
                                                          const Task* __restrict__ tasks_n,
                                                          const Sample2* __restrict__ samps, int parity,
                                                          long long n0) {
    constexpr int Q = stages_for(T, true);
    constexpr int STAGE_W = gen_stage_f4(true), STAGE_N = gen_stage_f4(true, 32 / NG_LANES);
    extern __shared__ float4 smem_f4[];
    __shared__ float4 coef_s[256];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int warps = blockDim.x >> 5;
    const bool narrow = (int)blockIdx.x >= nw_blocks;
    constexpr int PER_WARP = 32 / NG_LANES;
    const Task* first = narrow ? tasks_n + (size_t)(blockIdx.x - nw_blocks) * warps * PER_WARP
                               : tasks_w + (size_t)blockIdx.x * warps;
    if (first->scene < 0) return;
    const TmzDev* S = scenes + first->scene;
    for (int k = threadIdx.x; k < 256; k += blockDim.x) coef_s[k] = S->coef[k];
    __syncthreads();
    if (!narrow) {
        const Task tk = tasks_w[(size_t)blockIdx.x * warps + wib];
        if (tk.scene < 0) return;
        general_task<T, true, false, false, false>(S, tk, samps, parity, n0, coef_s,
                                                   smem_f4 + (size_t)wib * Q * STAGE_W, lane);
    } else {
        const Task* tw = first + (size_t)wib * PER_WARP;
        if (tw[0].scene < 0) return;   // a padding warp (whole warps only)
        const Task tk = tw[lane / NG_LANES];
        general_task<T, true, false, false, false, NG_LANES>(S, tk, samps, parity, n0, coef_s,
                                                             smem_f4 + (size_t)wib * Q * STAGE_N, lane);
    }
}

// ===========================================================================
// interior kernel: tasks with no CPML slab, design rectangle, source or probe in
// reach and all 120 output columns inside the grid (every other task runs the
// general kernel above).  Same wavefront; the steady-state loop body has no
// data-dependent branches.
// ===========================================================================
template <int T>
struct Ring {
    float4 E[T + 1], X[T + 2], Y[T + 1];
    uint32_t M[T + 1];
};

template <int T>
__device__ __forceinline__ void ring_shift_in(Ring<T>& R, const float4* st, int lane) {
#pragma unroll
    for (int k = T + 1; k >= 1; k--) R.X[k] = R.X[k - 1];
#pragma unroll
    for (int k = T; k >= 1; k--) {
        R.E[k] = R.E[k - 1];
        R.Y[k] = R.Y[k - 1];
        R.M[k] = R.M[k - 1];
    }
    R.E[0] = st[0 * 32 + lane];
    R.X[0] = st[1 * 32 + lane];
    R.Y[0] = st[2 * 32 + lane];
    R.M[0] = reinterpret_cast<const uint32_t*>(st + 3 * 32)[lane];
}

// one level t (H then E) on ring slot t; CT is the coefficient table's entry:
// float4 (Ca, Cb/dx, Cb/dy, Cb) or, for square cells, float2 (Ca, Cb/dx)
template <int T, typename CT>
__device__ __forceinline__ void level(Ring<T>& R, int t, float dbx, float dby, const CT* coef_s) {
    const float4 e = R.E[t], eu = R.E[t - 1];
    const float er = __shfl_down_sync(0xffffffffu, e.x, 1);
    R.X[t].x -= dby * (eu.x - e.x);
    R.X[t].y -= dby * (eu.y - e.y);
    R.X[t].z -= dby * (eu.z - e.z);
    R.X[t].w -= dby * (eu.w - e.w);
    R.Y[t].x += dbx * (e.y - e.x);
    R.Y[t].y += dbx * (e.z - e.y);
    R.Y[t].z += dbx * (e.w - e.z);
    R.Y[t].w += dbx * (er - e.w);
    const float4 y = R.Y[t];
    const float yl = __shfl_up_sync(0xffffffffu, y.w, 1);
    const uint32_t m = R.M[t];
    const CT c0 = coef_s[m & 255u], c1 = coef_s[(m >> 8) & 255u];
    const CT c2 = coef_s[(m >> 16) & 255u], c3 = coef_s[m >> 24];
    R.E[t].x = e_upd(e.x, y.x - yl, R.X[t].x - R.X[t + 1].x, c0);
    R.E[t].y = e_upd(e.y, y.y - y.x, R.X[t].y - R.X[t + 1].y, c1);
    R.E[t].z = e_upd(e.z, y.z - y.y, R.X[t].z - R.X[t + 1].z, c2);
    R.E[t].w = e_upd(e.w, y.w - y.z, R.X[t].w - R.X[t + 1].w, c3);
}

// One warp's interior task: T levels of the wavefront over the strip's rows,
// no boundary work.  coef_s is the scene's coefficient table (shared or global
// memory; float4 entries, or float2 (Ca, Cb/dx) for square cells), stage0 the
// warp's Q_I x stage_f4(false) float4 staging area.
template <int T, typename CT = float4>
__device__ __forceinline__ void interior_task(const TmzDev* __restrict__ S, const Task& tk, int parity,
                                              const CT* coef_s, float4* stage0, int lane) {
    constexpr int PF = pf_of(T, false);
    constexpr int SF4 = stage_f4(false);
    constexpr int Q = stages_for(T, false);
    static_assert((Q & (Q - 1)) == 0, "interior stage count must be a power of two");
    const int pitch = S->pitch;
    const float* __restrict__ ez_in = S->f[F_EZ][parity];
    const float* __restrict__ hx_in = S->f[F_HX][parity];
    const float* __restrict__ hy_in = S->f[F_HY][parity];
    float* __restrict__ ez_out = S->f[F_EZ][parity ^ 1];
    float* __restrict__ hx_out = S->f[F_HX][parity ^ 1];
    float* __restrict__ hy_out = S->f[F_HY][parity ^ 1];
    const uint8_t* __restrict__ mat = S->mat;
    const float dbx = S->dbx, dby = S->dby;

    const int cx = tk.x0 - HALO + 4 * lane;
    const int cs = cx + PAD_X;
    const bool out_lane = (lane >= HALO / 4) && (lane < 32 - HALO / 4) && (tk.xe == 0 || cx < tk.xe);
    const int s_row = tk.ya - T;
    const int r_last = tk.yb + T - 1;
    // rows past r_last are still inside the pad rows: the prefetch never needs a guard
    auto issue = [&](int row) {
        float4* st = stage0 + ((row - s_row) & (Q - 1)) * SF4;
        const size_t g = (size_t)(row + PAD_Y) * pitch + cs;
        cp_async16(st + 0 * 32 + lane, ez_in + g, true);
        cp_async16(st + 1 * 32 + lane, hx_in + g, true);
        cp_async16(st + 2 * 32 + lane, hy_in + g, true);
        cp_async4(reinterpret_cast<uint32_t*>(st + 3 * 32) + lane, mat + g);
    };

    Ring<T> R;
#pragma unroll
    for (int k = 0; k < T + 1; k++) {
        R.E[k] = make_float4(0, 0, 0, 0);
        R.Y[k] = R.E[k];
        R.M[k] = 0;
    }
#pragma unroll
    for (int k = 0; k < T + 2; k++) R.X[k] = make_float4(0, 0, 0, 0);
#pragma unroll
    for (int k = 0; k < PF; k++) {
        issue(s_row + k);
        cp_commit();
    }
    // Every level runs on every streamed row, also below the first one (on the
    // zero-initialised ring): those values are wrong but finite, and wrongness
    // climbs one row per level, so rows >= ya are exact after T levels.  The
    // first T steady rows are not stored.
    const int r_steady = tk.ya + T;
    for (int r = s_row; r <= r_last; ++r) {
        cp_wait<PF - 1>();
        ring_shift_in<T>(R, stage0 + ((r - s_row) & (Q - 1)) * SF4, lane);
#pragma unroll
        for (int t = 1; t <= T; t++) level<T, CT>(R, t, dbx, dby, coef_s);
        if (r >= r_steady) {
            const size_t g = (size_t)(r - T + PAD_Y) * pitch + cs;
            if (out_lane) {
                *reinterpret_cast<float4*>(ez_out + g) = R.E[T];
                *reinterpret_cast<float4*>(hx_out + g) = R.X[T];
                *reinterpret_cast<float4*>(hy_out + g) = R.Y[T];
            }
        }
        issue(r + PF);
        cp_commit();
    }
    cp_wait<0>();
}


// SQ: every scene has square cells, so the table is staged as (Ca, Cb/dx):
// half the shared-memory bandwidth of the lookups, which (four gathers per
// lane and level) share the pipe with the staging and the shuffles
template <int T, bool SQ>
__global__ void __launch_bounds__(256, 2) k_tmz_interior(const TmzDev* __restrict__ scenes,
                                                        const Task* __restrict__ tasks, int n_tasks,
                                                        int parity) {
    constexpr int SF4 = stage_f4(false);
    constexpr int Q = stages_for(T, false);
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
    interior_task<T, CT>(S, tk, parity, coef_s, smem_f4 + (size_t)wib * Q * SF4, lane);
}

// ---------------------------------------------------------------------------
// The same interior task with its rows brought in by the TMA engine
// (FDTD_OPT_BULK): per row one lane issues four cp.async.bulk copies -- the
// strip's 512 bytes of Ez, Hx and Hy and 144 bytes of material map around its
// 128 (the bulk copy wants a 16-byte aligned start) -- into a stage whose
// mbarrier counts the 1680 bytes, instead of four 16-byte cp.async per lane.
// The host uses it only where every interior task's field rows start on 16
// bytes and the material window stays inside the row.  Every mbarrier wait is
// bounded: past spin_limit polls the warp sets *err, waits for its copies in
// flight (bounded again, by at least 2^22 polls, so that no copy lands in
// shared memory the CTA has left) and returns; fdtd_sync reports
// FDTD_ETIMEOUT.
// ---------------------------------------------------------------------------
constexpr int BULK_FIELD_BYTES = STRIP * 4;                  // 512
constexpr int BULK_MAT_BYTES = STRIP + 16;                   // 144: 128 bytes from any start
constexpr int BULK_STAGE_BYTES = 3 * BULK_FIELD_BYTES + BULK_MAT_BYTES;   // 1680
constexpr int BULK_STAGE_F4 = BULK_STAGE_BYTES / 16;         // 105
static_assert(BULK_STAGE_BYTES % 16 == 0, "a bulk stage must keep every copy 16-byte aligned");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
// true once the phase of the given parity has completed
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
// bounded wait; false when it gave up
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
    for (long long k = 0; k < limit; k++)
        if (mbar_try(bar, parity)) return true;
    return false;
}

template <int T, typename CT>
__device__ __forceinline__ void interior_task_bulk(const TmzDev* __restrict__ S, const Task& tk, int parity,
                                                   const CT* coef_s, float4* stage0, uint64_t* bars, int lane,
                                                   long long spin_limit, int* err) {
    constexpr int PF = pf_of(T, false);
    constexpr int Q = stages_for(T, false);
    static_assert((Q & (Q - 1)) == 0, "interior stage count must be a power of two");
    const int pitch = S->pitch;
    const float* __restrict__ ez_in = S->f[F_EZ][parity];
    const float* __restrict__ hx_in = S->f[F_HX][parity];
    const float* __restrict__ hy_in = S->f[F_HY][parity];
    float* __restrict__ ez_out = S->f[F_EZ][parity ^ 1];
    float* __restrict__ hx_out = S->f[F_HX][parity ^ 1];
    float* __restrict__ hy_out = S->f[F_HY][parity ^ 1];
    const uint8_t* __restrict__ mat = S->mat;
    const float dbx = S->dbx, dby = S->dby;

    const int cs0 = tk.x0 - HALO + PAD_X;          // first loaded column (16-byte aligned field rows)
    const int m0 = cs0 & ~15, moff = cs0 - m0;     // material window start and the strip's offset in it
    const int cs = cs0 + 4 * lane;
    const bool out_lane = (lane >= HALO / 4) && (lane < 32 - HALO / 4) && (tk.xe == 0 || cs - PAD_X < tk.xe);
    const int s_row = tk.ya - T;
    const int r_last = tk.yb + T - 1;
    const uint32_t bar0 = smem_u32(bars);
    if (lane == 0)
        for (int k = 0; k < Q; k++) mbar_init(bar0 + 8 * k);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    __syncwarp();
    // rows past r_last are still inside the pad rows: the prefetch never needs a guard
    auto issue = [&](int row) {
        __syncwarp();   // every lane has read the stage's previous row
        if (lane == 0) {
            const int k = (row - s_row) & (Q - 1);
            const uint32_t st = smem_u32(stage0 + (size_t)k * BULK_STAGE_F4), bar = bar0 + 8 * k;
            const size_t g = (size_t)(row + PAD_Y) * pitch;
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            mbar_expect(bar, BULK_STAGE_BYTES);
            bulk_g2s(st, ez_in + g + cs0, BULK_FIELD_BYTES, bar);
            bulk_g2s(st + BULK_FIELD_BYTES, hx_in + g + cs0, BULK_FIELD_BYTES, bar);
            bulk_g2s(st + 2 * BULK_FIELD_BYTES, hy_in + g + cs0, BULK_FIELD_BYTES, bar);
            bulk_g2s(st + 3 * BULK_FIELD_BYTES, mat + g + m0, BULK_MAT_BYTES, bar);
        }
    };

    Ring<T> R;
#pragma unroll
    for (int k = 0; k < T + 1; k++) {
        R.E[k] = make_float4(0, 0, 0, 0);
        R.Y[k] = R.E[k];
        R.M[k] = 0;
    }
#pragma unroll
    for (int k = 0; k < T + 2; k++) R.X[k] = make_float4(0, 0, 0, 0);
    for (int k = 0; k < PF; k++) issue(s_row + k);
    const int r_steady = tk.ya + T;
    bool ok = true;
    int r = s_row;
    for (; r <= r_last; ++r) {
        const int u = r - s_row, k = u & (Q - 1);
        if (!mbar_wait(bar0 + 8 * k, (uint32_t)(u / Q) & 1u, spin_limit)) {
            ok = false;
            break;
        }
        const float4* st = stage0 + (size_t)k * BULK_STAGE_F4;
        // shift the ring: the staged row enters at slot 0 (field rows at 0, 32,
        // 64 float4; the material row 4 bytes per lane from its offset)
#pragma unroll
        for (int q = T + 1; q >= 1; q--) R.X[q] = R.X[q - 1];
#pragma unroll
        for (int q = T; q >= 1; q--) {
            R.E[q] = R.E[q - 1];
            R.Y[q] = R.Y[q - 1];
            R.M[q] = R.M[q - 1];
        }
        R.E[0] = st[0 * 32 + lane];
        R.X[0] = st[1 * 32 + lane];
        R.Y[0] = st[2 * 32 + lane];
        R.M[0] = *reinterpret_cast<const uint32_t*>(reinterpret_cast<const uint8_t*>(st + 3 * 32) + moff + 4 * lane);
#pragma unroll
        for (int t = 1; t <= T; t++) level<T, CT>(R, t, dbx, dby, coef_s);
        if (r >= r_steady) {
            const size_t g = (size_t)(r - T + PAD_Y) * pitch + cs;
            if (out_lane) {
                *reinterpret_cast<float4*>(ez_out + g) = R.E[T];
                *reinterpret_cast<float4*>(hx_out + g) = R.X[T];
                *reinterpret_cast<float4*>(hy_out + g) = R.Y[T];
            }
        }
        issue(r + PF);
    }
    // drain: every copy issued and not yet consumed lands before the warp leaves
    // (rows r .. r - 1 + PF: the last row issued, whether the loop finished or
    // gave up at row r; bounded waits)
    const long long drain_limit = spin_limit > (1ll << 22) ? spin_limit : (1ll << 22);
    for (int q = r; q <= r - 1 + PF; q++) {
        const int u = q - s_row;
        if (!mbar_wait(bar0 + 8 * (u & (Q - 1)), (uint32_t)(u / Q) & 1u, drain_limit)) ok = false;
    }
    if (!ok && lane == 0) atomicExch(err, 1);
}

// interior kernel with bulk row copies; the dynamic shared memory holds each
// warp's Q_I stages of BULK_STAGE_BYTES, then each warp's Q_I mbarriers
template <int T, bool SQ>
__global__ void __launch_bounds__(256, 2) k_tmz_interior_bulk(const TmzDev* __restrict__ scenes,
                                                             const Task* __restrict__ tasks, int n_tasks,
                                                             int parity, long long spin_limit, int* err) {
    constexpr int Q = stages_for(T, false);
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
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_f4 + (size_t)warps * Q * BULK_STAGE_F4) + (size_t)wib * Q;
    interior_task_bulk<T, CT>(S, tk, parity, coef_s, smem_f4 + (size_t)wib * Q * BULK_STAGE_F4, bars, lane,
                              spin_limit, err);
}

// ===========================================================================
// persistent kernel: one cooperative launch advances every scene of a batch
// by n_blocks * T steps.  The work is a list of items per T-step block -- an
// interior task, a whole-warp general task (CPML, design, source, probes) or
// four narrow x-slab tasks -- and warps pull (block, item) pairs in order from
// a counter, so uneven scene sizes balance themselves.  There is no barrier
// between blocks: an item of block b waits only until every item whose region
// it reads or overwrites (its neighbours, itself included) has finished block
// b - 1, as counted in done[] (block b reads buffer p and writes 1 - p, so these
// are the only items whose data it touches).  Every wait is bounded: after
// spin_limit polls the warp sets the error flag and returns, and the others
// stop waiting when they see it.
//
// The CTA is 12 warps in two classes, as the items need registers: warps 0-7
// take interior items and give registers back (setmaxnreg down to 128, what
// the interior wavefront needs), warps 8-11 take general and narrow items and
// get them (up to 248).  The split spends exactly the 384 x 168 registers the
// CTA is launched with (the host checks the kernel's count before launching,
// since a larger split would wait forever).  Each class pulls from its own
// queue in (block, space) order; both are served in block order and every item
// waits only for the previous block, so the lowest unfinished block always
// progresses.
//
// ctl layout (unsigned): [0] next interior (block, item) index, [1] next
// general one, [2] error flag (kept by the host until fdtd_sync reports it).
// stall_item >= 0 names an item that never reports block 0 done (a test of the
// timeout path); -1 in normal runs.
// ===========================================================================
constexpr int PW_INT = 8, PW_GEN = 4;                 // warps per class
constexpr int PREG_LAUNCH = 168, PREG_INT = 128, PREG_GEN = 248;
static_assert(PW_INT * PREG_INT + PW_GEN * PREG_GEN <= (PW_INT + PW_GEN) * PREG_LAUNCH,
              "the register split must fit the CTA's launch allocation");

template <int T>
__host__ __device__ constexpr int pstage_int() { return stages_for(T, false) * stage_f4(false); }
template <int T>
__host__ __device__ constexpr int pstage_gen() { return stages_for(T, true) * gen_stage_f4(true, 32 / NG_LANES); }

// one warp's loop over its class's queue: claim, wait for the neighbours'
// previous block, run, publish (general warps lending a hand with interior
// items measured no faster on the 64-scene batch: 539 vs 545 G)
template <int T, bool WREC, bool GEN>
__device__ __forceinline__ void persistent_loop(const TmzDev* __restrict__ scenes, const Task* __restrict__ ptasks,
                                                const int2* __restrict__ items, const int* __restrict__ queue,
                                                int n_int, int n_gen, const int* __restrict__ dep_off,
                                                const int* __restrict__ dep_idx, const Sample2* __restrict__ samps,
                                                int parity0, long long n0, int n_blocks, unsigned* ctl,
                                                unsigned* done, long long spin_limit, int stall_item, float4* stage0,
                                                int lane) {
    volatile int* verr = reinterpret_cast<volatile int*>(ctl + 2);
    // an earlier launch of this context timed out and nobody has read the flag yet
    if (*verr) return;
    const long long tot_i = (long long)n_blocks * n_int, tot_g = (long long)n_blocks * n_gen;
    for (;;) {
        constexpr int sel = GEN ? 1 : 0;   // the general queue follows the interior one
        const long long tot = GEN ? tot_g : tot_i;
        long long idx = 0;
        if (lane == 0) idx = (long long)atomicAdd(ctl + sel, 1u);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= tot) return;
        const int nq = GEN ? n_gen : n_int;
        const int b = (int)(idx / nq), it = queue[(GEN ? n_int : 0) + (int)(idx % nq)];
        // wait for the neighbours' block b - 1: the lanes poll up to 32 counts at
        // once (relaxed loads), then one fence orders the item's reads after them
        if (b > 0) {
            const int d0 = dep_off[it], nd = dep_off[it + 1] - d0;
            long long spins = 0;
            for (int base = 0; base < nd; base += 32) {
                const int q = base + lane;
                const unsigned* d = q < nd ? done + dep_idx[d0 + q] : nullptr;
                for (;;) {
                    int ready = 1;
                    if (d) {
                        unsigned v;
                        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(d) : "memory");
                        ready = v >= (unsigned)b;
                    }
                    if (__all_sync(0xffffffffu, ready)) break;
                    if (__any_sync(0xffffffffu, *verr != 0) || ++spins > spin_limit) {
                        if (lane == 0) atomicExch(reinterpret_cast<int*>(ctl + 2), 1);
                        return;
                    }
                    __nanosleep(100);
                }
            }
            __threadfence();
        }
        __syncwarp();
        const int parity = parity0 ^ (b & 1);
        const long long nb = n0 + (long long)b * T;
        const int2 item = items[it];
        if constexpr (GEN) {
            if (item.x == PITEM_NARROW) {
                const Task tk = ptasks[item.y + lane / NG_LANES];
                const TmzDev* S = scenes + tk.scene;
                general_task<T, true, false, false, false, NG_LANES>(S, tk, samps, parity, nb, S->coef, stage0, lane);
            } else {
                const Task tk = ptasks[item.y];
                const TmzDev* S = scenes + tk.scene;
                general_task<T, true, false, WREC>(S, tk, samps, parity, nb, S->coef, stage0, lane);
            }
        } else {
            const Task tk = ptasks[item.y];
            const TmzDev* S = scenes + tk.scene;
            interior_task<T>(S, tk, parity, S->coef, stage0, lane);
        }
        // publish: every lane's stores of this item, then the count
        __syncwarp();
        if (lane == 0 && !(b == 0 && it == stall_item)) {
            __threadfence();   // release: the fence, then a plain store of the count
            asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(done + it), "r"((unsigned)(b + 1)) : "memory");
        }
    }
}

template <int T, bool WREC>
__global__ void __launch_bounds__((PW_INT + PW_GEN) * 32, 1) k_tmz_persistent(
    const TmzDev* __restrict__ scenes, const Task* __restrict__ ptasks, const int2* __restrict__ items,
    const int* __restrict__ queue, int n_int, int n_gen, const int* __restrict__ dep_off,
    const int* __restrict__ dep_idx, const Sample2* __restrict__ samps, int parity0, long long n0, int n_blocks,
    unsigned* ctl, unsigned* done, long long spin_limit, int stall_item) {
    extern __shared__ float4 smem_f4[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    if (wib >= PW_INT) {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(PREG_GEN) : "memory");
        float4* stage0 = smem_f4 + (size_t)PW_INT * pstage_int<T>() + (size_t)(wib - PW_INT) * pstage_gen<T>();
        persistent_loop<T, WREC, true>(scenes, ptasks, items, queue, n_int, n_gen, dep_off, dep_idx, samps, parity0,
                                       n0, n_blocks, ctl, done, spin_limit, stall_item, stage0, lane);
    } else {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(PREG_INT) : "memory");
        float4* stage0 = smem_f4 + (size_t)wib * pstage_int<T>();
        persistent_loop<T, WREC, false>(scenes, ptasks, items, queue, n_int, n_gen, dep_off, dep_idx, samps, parity0,
                                        n0, n_blocks, ctl, done, spin_limit, stall_item, stage0, lane);
    }
}

// Second layout (FDTD_OPT_PLAYOUT = k > 0): 16-warp CTAs of two kinds, so
// that most SMs hold 16 interior warps as the per-block launches do.  The first
// k CTAs run general and narrow items: warpgroups 0 and 1 take registers up to
// 232 (setmaxnreg.inc), warpgroups 2 and 3 give theirs back down to 24 and
// return, which balances the CTA's 512 x 128 launch registers exactly (and each
// SM sub-partition's share: every warpgroup has one warp on each).  The other
// CTAs run 16 interior warps at the launch's 128 registers.  Both kinds take
// items from the same two ordered queues as the first layout.
constexpr int PW2_WARPS = 16, PREG2_LAUNCH = 128, PREG2_GEN = 232, PREG2_IDLE = 24;
static_assert(8 * PREG2_GEN + 8 * PREG2_IDLE == PW2_WARPS * PREG2_LAUNCH,
              "the wide layout's register split must spend exactly the CTA's launch allocation");

template <int T, bool WREC>
__global__ void __launch_bounds__(PW2_WARPS * 32, 1) k_tmz_persistent_wide(
    const TmzDev* __restrict__ scenes, const Task* __restrict__ ptasks, const int2* __restrict__ items,
    const int* __restrict__ queue, int n_int, int n_gen, const int* __restrict__ dep_off,
    const int* __restrict__ dep_idx, const Sample2* __restrict__ samps, int parity0, long long n0, int n_blocks,
    unsigned* ctl, unsigned* done, long long spin_limit, int stall_item, int n_gcta) {
    extern __shared__ float4 smem_f4[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    if ((int)blockIdx.x < n_gcta) {
        if (wib >= 8) {
            asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(PREG2_IDLE) : "memory");
            return;
        }
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(PREG2_GEN) : "memory");
        float4* stage0 = smem_f4 + (size_t)wib * pstage_gen<T>();
        persistent_loop<T, WREC, true>(scenes, ptasks, items, queue, n_int, n_gen, dep_off, dep_idx, samps, parity0,
                                       n0, n_blocks, ctl, done, spin_limit, stall_item, stage0, lane);
    } else {
        float4* stage0 = smem_f4 + (size_t)wib * pstage_int<T>();
        persistent_loop<T, WREC, false>(scenes, ptasks, items, queue, n_int, n_gen, dep_off, dep_idx, samps, parity0,
                                        n0, n_blocks, ctl, done, spin_limit, stall_item, stage0, lane);
    }
}

// dynamic shared memory of the persistent kernel: the interior warps' staging,
// then the general warps'
static size_t persistent_smem(int T) {
    const size_t i = (size_t)stages_for(T, false) * stage_f4(false);
    const size_t g = (size_t)stages_for(T, true) * gen_stage_f4(true, 32 / NG_LANES);
    return ((size_t)PW_INT * i + (size_t)PW_GEN * g) * sizeof(float4);
}

template <int T, bool WREC>
static cudaError_t launch_persistent_T(const fdtd_ctx* c, cudaStream_t st, int parity, long long n0, int n_blocks,
                                       long long spin_limit, int* grid_out) {
    const int threads = (PW_INT + PW_GEN) * 32;
    const size_t smem = persistent_smem(T);
    cudaError_t e = ensure_dyn_smem((const void*)k_tmz_persistent<T, WREC>, smem);
    if (e != cudaSuccess) return e;
    // the register split is exact only for a kernel built at PREG_LAUNCH
    // registers; any other count could leave setmaxnreg.inc waiting forever
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, (const void*)k_tmz_persistent<T, WREC>);
    if (e != cudaSuccess) return e;
    if (fa.numRegs != PREG_LAUNCH) return cudaErrorInvalidConfiguration;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tmz_persistent<T, WREC>, threads, smem);
    if (e != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = per_sm * sms;
    *grid_out = grid;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // every CTA resident: a waited-on item is always being worked
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_tmz_persistent<T, WREC>, (const TmzDev*)c->d_scenes, (const Task*)c->d_ptasks,
                              (const int2*)c->d_pitems, (const int*)c->d_pq, c->n_pint, c->n_pgen,
                              (const int*)c->d_dep_off, (const int*)c->d_dep_idx, (const Sample2*)c->d_samp, parity,
                              n0, n_blocks, c->d_ctl, c->d_done, spin_limit, c->opt_debug_skip);
}

// the wide layout: grid = one 16-warp CTA per SM, the first n_gcta of them for
// general items (at least one CTA of each kind)
template <int T, bool WREC>
static cudaError_t launch_persistent_wide_T(const fdtd_ctx* c, cudaStream_t st, int parity, long long n0,
                                            int n_blocks, long long spin_limit, int n_gcta, int* grid_out) {
    const int threads = PW2_WARPS * 32;
    const size_t smem = std::max((size_t)PW2_WARPS * pstage_int<T>(), (size_t)8 * pstage_gen<T>()) * sizeof(float4);
    cudaError_t e = ensure_dyn_smem((const void*)k_tmz_persistent_wide<T, WREC>, smem);
    if (e != cudaSuccess) return e;
    // the register split is exact only for a kernel built at PREG2_LAUNCH
    // registers; any other count could leave setmaxnreg.inc waiting forever
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, (const void*)k_tmz_persistent_wide<T, WREC>);
    if (e != cudaSuccess) return e;
    if (fa.numRegs != PREG2_LAUNCH) return cudaErrorInvalidConfiguration;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tmz_persistent_wide<T, WREC>, threads, smem);
    if (e != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = per_sm * sms;
    const int ng = std::min(std::max(n_gcta, 1), grid - 1);
    *grid_out = grid;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // every CTA resident: a waited-on item is always being worked
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_tmz_persistent_wide<T, WREC>, (const TmzDev*)c->d_scenes,
                              (const Task*)c->d_ptasks, (const int2*)c->d_pitems, (const int*)c->d_pq, c->n_pint,
                              c->n_pgen, (const int*)c->d_dep_off, (const int*)c->d_dep_idx,
                              (const Sample2*)c->d_samp, parity, n0, n_blocks, c->d_ctl, c->d_done, spin_limit,
                              c->opt_debug_skip, ng);
}

int tmz_persistent_launch(fdtd_ctx* c, int T, long long n0, int n_blocks, int parity) {
    cudaError_t e = cudaMemsetAsync(c->d_ctl, 0, 2 * sizeof(unsigned), c->stream);
    if (e == cudaSuccess && c->n_pitems > 0)
        e = cudaMemsetAsync(c->d_done, 0, (size_t)c->n_pitems * sizeof(unsigned), c->stream);
    int grid = 0;
    const bool wrec = adj_edge_mode(c);   // edge-weight reverse mode: keep the design window
    // the wide layout has builds for T = 2..4 without the window writes
    const int ng = (T >= 2 && !wrec) ? c->opt_playout : 0;
    const long long sl = c->spin_limit;
    if (e == cudaSuccess && c->n_pitems > 0 && ng > 0) {
        switch (T) {
            case 2: e = launch_persistent_wide_T<2, false>(c, c->stream, parity, n0, n_blocks, sl, ng, &grid); break;
            case 3: e = launch_persistent_wide_T<3, false>(c, c->stream, parity, n0, n_blocks, sl, ng, &grid); break;
            default: e = launch_persistent_wide_T<4, false>(c, c->stream, parity, n0, n_blocks, sl, ng, &grid); break;
        }
    } else if (e == cudaSuccess && c->n_pitems > 0) {
        switch (T) {
            case 1: e = wrec ? launch_persistent_T<1, true>(c, c->stream, parity, n0, n_blocks, c->spin_limit, &grid)
                             : launch_persistent_T<1, false>(c, c->stream, parity, n0, n_blocks, c->spin_limit, &grid);
                break;
            case 2: e = wrec ? launch_persistent_T<2, true>(c, c->stream, parity, n0, n_blocks, c->spin_limit, &grid)
                             : launch_persistent_T<2, false>(c, c->stream, parity, n0, n_blocks, c->spin_limit, &grid);
                break;
            case 3: e = wrec ? launch_persistent_T<3, true>(c, c->stream, parity, n0, n_blocks, c->spin_limit, &grid)
                             : launch_persistent_T<3, false>(c, c->stream, parity, n0, n_blocks, c->spin_limit, &grid);
                break;
            default: e = wrec ? launch_persistent_T<4, true>(c, c->stream, parity, n0, n_blocks, c->spin_limit, &grid)
                              : launch_persistent_T<4, false>(c, c->stream, parity, n0, n_blocks, c->spin_limit, &grid);
                break;
        }
    }
    c->launches++;
    c->opt_debug_skip = -1;   // the test hook covers one launch
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_err, c->d_ctl + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("persistent launch: ") + cudaGetErrorString(e);
        return FDTD_ECUDA;
    }
    return FDTD_OK;
}

// ===========================================================================
// unfused pair: one H launch, one E launch, one source/record launch per step
// ===========================================================================
__global__ void k_tmz_h(const TmzDev* __restrict__ scenes, int parity) {
    const TmzDev& S = scenes[blockIdx.z];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= S.nx || j >= S.ny) return;
    const int pitch = S.pitch;
    const size_t c = sidx(pitch, i, j);
    const float* ez = S.f[F_EZ][parity];
    const float e = ez[c];
    float dey = ez[c + pitch] - e;   // row ny is a zero pad row: ghost PEC
    float dex = ez[c + 1] - e;       // column nx is a zero pad column
    if (S.has_pml) {
        const Prof pr{S.prof, pitch, S.rows};
        const int rs = j + PAD_Y, cs = i + PAD_X;
        const float by = pr.bHy(rs), cy = pr.cHy(rs);
        if (by != 0.f || cy != 0.f) {
            float* p = S.f[F_PHXY][parity];
            const float v = by * p[c] + cy * dey;
            p[c] = v;
            dey += v;
        }
        const float bx = pr.bHx(cs), cxx = pr.cHx(cs);
        if (bx != 0.f || cxx != 0.f) {
            float* p = S.f[F_PHYX][parity];
            const float v = bx * p[c] + cxx * dex;
            p[c] = v;
            dex += v;
        }
    }
    if (S.split) {
        // split-field layer (Sec. III-C): H damped by sigma* of the axis its
        // derivative runs along, semi-implicit as eq. (7)
        const Prof pr{S.prof, pitch, S.rows};
        const int np = S.split;
        float* hx = S.f[F_HX][parity];
        float* hy = S.f[F_HY][parity];
        if (j < np || j >= S.ny - np) hx[c] = pr.bHy(j + PAD_Y) * hx[c] - pr.cHy(j + PAD_Y) * dey;
        else hx[c] -= S.dby * dey;
        if (i < np || i >= S.nx - np) hy[c] = pr.bHx(i + PAD_X) * hy[c] + pr.cHx(i + PAD_X) * dex;
        else hy[c] += S.dbx * dex;
        return;
    }
    S.f[F_HX][parity][c] -= S.dby * dey;
    S.f[F_HY][parity][c] += S.dbx * dex;
}

__global__ void k_tmz_e(const TmzDev* __restrict__ scenes, int parity) {
    const TmzDev& S = scenes[blockIdx.z];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= S.nx || j >= S.ny) return;
    const int pitch = S.pitch;
    const size_t c = sidx(pitch, i, j);
    const float* hx = S.f[F_HX][parity];
    const float* hy = S.f[F_HY][parity];
    float dhy = hy[c] - hy[c - 1];
    float dhx = hx[c] - hx[c - pitch];
    if (S.has_pml) {
        const Prof pr{S.prof, pitch, S.rows};
        const int rs = j + PAD_Y, cs = i + PAD_X;
        const float bx = pr.bEx(cs), cxx = pr.cEx(cs);
        if (bx != 0.f || cxx != 0.f) {
            float* p = S.f[F_PEZX][parity];
            const float v = bx * p[c] + cxx * dhy;
            p[c] = v;
            dhy += v;
        }
        const float by = pr.bEy(rs), cy = pr.cEy(rs);
        if (by != 0.f || cy != 0.f) {
            float* p = S.f[F_PEZY][parity];
            const float v = by * p[c] + cy * dhx;
            p[c] = v;
            dhx += v;
        }
    }
    float4 co = S.coef[S.mat[c]];
    if (S.dsg_w > 0) {
        const int di = i - S.dsg_i0, dj = j - S.dsg_j0;
        if (di >= 0 && di < S.dsg_w && dj >= 0 && dj < S.dsg_h) co = S.dsg_coef[(size_t)dj * S.dsg_w + di];
    }
    float* ez = S.f[F_EZ][parity];
    if (S.split && i >= 1 && j >= 1) {
        const int np = S.split;
        const bool lx = i < np || i > S.nx - np, ly = j < np || j > S.ny - np;
        if (lx || ly) {
            // split-field layer (Sec. III-C): Ez = Ezx + Ezy, Ezy kept in the
            // psi_Ezy array, each part damped along its own axis (vacuum cells)
            const Prof pr{S.prof, pitch, S.rows};
            float* pzy = S.f[F_PEZY][parity];
            const float ezy0 = pzy[c], ezx0 = ez[c] - ezy0;
            const float ax = lx ? pr.bEx(i + PAD_X) : co.x, bx = lx ? pr.cEx(i + PAD_X) : co.y;
            const float ay = ly ? pr.bEy(j + PAD_Y) : co.x, by = ly ? pr.cEy(j + PAD_Y) : co.z;
            const float ezx = ax * ezx0 + bx * dhy;
            const float ezy = ay * ezy0 - by * dhx;
            pzy[c] = ezy;
            ez[c] = ezx + ezy;
            return;
        }
    }
    ez[c] = e_upd(ez[c], dhy, dhx, co);
}

__global__ void k_tmz_src_rec(const TmzDev* __restrict__ scenes, const Sample2* __restrict__ samps,
                              const int* __restrict__ samp_off, int parity, long long n) {
    const TmzDev& S = scenes[blockIdx.x];
    if (S.src_i >= 0 && n < S.src_len)
        for (int j = S.src_j + (int)threadIdx.x; j < S.src_j1; j += blockDim.x)
            S.f[F_EZ][parity][sidx(S.pitch, S.src_i, j)] += S.src_wave[n];
    __syncthreads();
    for (int q = samp_off[blockIdx.x] + threadIdx.x; q < samp_off[blockIdx.x + 1]; q += blockDim.x) {
        const Sample2 sp = samps[q];
        const int f = sp.comp == 0 ? F_EZ : (sp.comp == 1 ? F_HX : F_HY);
        S.rec[n * S.n_rec + sp.slot] = S.f[f][parity][sidx(S.pitch, sp.i, sp.j)];
    }
}

// ===========================================================================
// running DFT of recorded samples, compensated FP32
// ===========================================================================
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

__global__ void k_dft_cells(const float* __restrict__ rec, int n_rec, int slot0, int n_cells,
                            const double* __restrict__ freq, int n_freq, double dt, float4* acc,
                            long long n0, int nsteps) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n_cells * n_freq) return;
    const int cell = id / n_freq, f = id % n_freq;
    float4 a = acc[id];
    const double fdt = freq[f] * dt;
    const float fdtf = (float)dt;
    for (int k = 0; k < nsteps; k++) {
        const long long n = n0 + k;
        const float e = rec[n * n_rec + slot0 + cell];
        double ph = fdt * (double)(n + 1);
        ph -= floor(ph);
        double sn, cs;
        sincospi(2.0 * ph, &sn, &cs);
        kahan_add(a.x, a.z, e * ((float)cs * fdtf));
        kahan_add(a.y, a.w, -e * ((float)sn * fdtf));
    }
    acc[id] = a;
}

__global__ void k_tmz_finite(const TmzDev* __restrict__ scenes, int parity, int* bad) {
    const TmzDev& S = scenes[blockIdx.z];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= S.nx || j >= S.ny) return;
    const size_t c = sidx(S.pitch, i, j);
    const float v = S.f[F_EZ][parity][c] + S.f[F_HX][parity][c] + S.f[F_HY][parity][c];
    if (!isfinite(v)) atomicOr(bad, 1);
}

// ===========================================================================
// launchers
// ===========================================================================
// variant 0: interior (clean) tasks; 1: CPML tasks; 2: lite tasks (design
// rectangle, source, probes or ragged edge, no CPML); 3: split-field layer
// tasks; 5, 6: variants 1, 2 keeping the design window (edge-weight mode);
// 7: variant 1 compiled without the design paths (CPML tasks with no design in
// reach; those with one run variant 1 or 5)
template <int T, int V>
static cudaError_t launch_fused_T(const Task* tasks, int n_tasks, int warps, const fdtd_ctx* c, cudaStream_t st,
                                  long long n0, int parity) {
    const size_t smem = tmz_fused_smem(T, warps, V);
    const int blocks = n_tasks / warps;   // task lists are padded to whole CTAs
    cudaError_t e;
    if (V == 1) {
        e = ensure_dyn_smem((const void*)k_tmz_fused<T, true>, smem);
        if (e != cudaSuccess) return e;
        k_tmz_fused<T, true><<<blocks, warps * 32, smem, st>>>(c->d_scenes, tasks, n_tasks, c->d_samp, parity, n0);
    } else if (V == 7) {
        e = ensure_dyn_smem((const void*)k_tmz_fused<T, true, false, false, false>, smem);
        if (e != cudaSuccess) return e;
        k_tmz_fused<T, true, false, false, false><<<blocks, warps * 32, smem, st>>>(c->d_scenes, tasks, n_tasks,
                                                                                     c->d_samp, parity, n0);
    } else if (V == 5) {
        e = ensure_dyn_smem((const void*)k_tmz_fused<T, true, false, true>, smem);
        if (e != cudaSuccess) return e;
        k_tmz_fused<T, true, false, true><<<blocks, warps * 32, smem, st>>>(c->d_scenes, tasks, n_tasks, c->d_samp,
                                                                             parity, n0);
    } else if (V == 6) {
        e = ensure_dyn_smem((const void*)k_tmz_fused<T, false, false, true>, smem);
        if (e != cudaSuccess) return e;
        k_tmz_fused<T, false, false, true><<<blocks, warps * 32, smem, st>>>(c->d_scenes, tasks, n_tasks, c->d_samp,
                                                                              parity, n0);
    } else if (V == 3) {
        e = ensure_dyn_smem((const void*)k_tmz_fused<T, true, true>, smem);
        if (e != cudaSuccess) return e;
        k_tmz_fused<T, true, true><<<blocks, warps * 32, smem, st>>>(c->d_scenes, tasks, n_tasks, c->d_samp, parity,
                                                                      n0);
    } else if (V == 2) {
        e = ensure_dyn_smem((const void*)k_tmz_fused<T, false>, smem);
        if (e != cudaSuccess) return e;
        k_tmz_fused<T, false><<<blocks, warps * 32, smem, st>>>(c->d_scenes, tasks, n_tasks, c->d_samp, parity, n0);
    } else if (c->use_bulk) {
        const size_t sm = (size_t)warps * stages_for(T, false) * (BULK_STAGE_BYTES + 8);
        if (c->coef_sq) {
            e = ensure_dyn_smem((const void*)k_tmz_interior_bulk<T, true>, sm);
            if (e != cudaSuccess) return e;
            k_tmz_interior_bulk<T, true><<<blocks, warps * 32, sm, st>>>(c->d_scenes, tasks, n_tasks, parity,
                                                                           c->spin_limit, c->d_bulk_err);
        } else {
            e = ensure_dyn_smem((const void*)k_tmz_interior_bulk<T, false>, sm);
            if (e != cudaSuccess) return e;
            k_tmz_interior_bulk<T, false><<<blocks, warps * 32, sm, st>>>(c->d_scenes, tasks, n_tasks, parity,
                                                                            c->spin_limit, c->d_bulk_err);
        }
    } else if (c->coef_sq) {
        e = ensure_dyn_smem((const void*)k_tmz_interior<T, true>, smem);
        if (e != cudaSuccess) return e;
        k_tmz_interior<T, true><<<blocks, warps * 32, smem, st>>>(c->d_scenes, tasks, n_tasks, parity);
    } else {
        e = ensure_dyn_smem((const void*)k_tmz_interior<T, false>, smem);
        if (e != cudaSuccess) return e;
        k_tmz_interior<T, false><<<blocks, warps * 32, smem, st>>>(c->d_scenes, tasks, n_tasks, parity);
    }
    return cudaGetLastError();
}

template <int T>
static cudaError_t launch_cpml_mixed_T(const fdtd_ctx* c, cudaStream_t st, long long n0, int parity) {
    const int warps = c->warps_b;
    const size_t smem = tmz_fused_smem(T, warps, 8);   // the larger stage of the two task kinds
    const int nw = c->n_tasks_b / warps, nn = c->n_tasks_n / (warps * 32 / NG_LANES);
    cudaError_t e = ensure_dyn_smem((const void*)k_tmz_cpml_mixed<T>, smem);
    if (e != cudaSuccess) return e;
    k_tmz_cpml_mixed<T><<<nw + nn, warps * 32, smem, st>>>(c->d_scenes, c->d_tasks_b, nw, c->d_tasks_n, c->d_samp,
                                                           parity, n0);
    return cudaGetLastError();
}

static cudaError_t launch_cpml_mixed(const fdtd_ctx* c, cudaStream_t st, int T, long long n0, int parity) {
    switch (T) {
        case 1: return launch_cpml_mixed_T<1>(c, st, n0, parity);
        case 2: return launch_cpml_mixed_T<2>(c, st, n0, parity);
        case 3: return launch_cpml_mixed_T<3>(c, st, n0, parity);
        case 4: return launch_cpml_mixed_T<4>(c, st, n0, parity);
    }
    return cudaErrorInvalidValue;
}

template <int V>
static cudaError_t launch_fused(const Task* tasks, int n_tasks, int warps, const fdtd_ctx* c, cudaStream_t st, int T,
                                long long n0, int parity) {
    switch (T) {
        case 1: return launch_fused_T<1, V>(tasks, n_tasks, warps, c, st, n0, parity);
        case 2: return launch_fused_T<2, V>(tasks, n_tasks, warps, c, st, n0, parity);
        case 3: return launch_fused_T<3, V>(tasks, n_tasks, warps, c, st, n0, parity);
        case 4: return launch_fused_T<4, V>(tasks, n_tasks, warps, c, st, n0, parity);
    }
    return cudaErrorInvalidValue;
}

// one T-step block: interior tasks on the context's stream, CPML and lite tasks
// on two forked streams, joined before the next block reads the new buffer
int tmz_fused_launch(fdtd_ctx* c, int T, int warps, long long n0, int parity) {
    cudaError_t e = cudaSuccess;
    const int nb = c->n_tasks_b + c->n_tasks_s + c->n_tasks_bd + c->n_tasks_n, nl = c->n_tasks_l, ni = c->n_tasks;
    cudaStream_t sb = c->stream, sl = c->stream;
    if ((nb > 0) + (nl > 0) + (ni > 0) > 1) {
        e = cudaEventRecord(c->ev_fork, c->stream);
        if (e == cudaSuccess && nb > 0) {
            e = cudaStreamWaitEvent(c->aux, c->ev_fork, 0);
            sb = c->aux;
        }
        if (e == cudaSuccess && nl > 0) {
            e = cudaStreamWaitEvent(c->aux2, c->ev_fork, 0);
            sl = c->aux2;
        }
    }
    // edge-weight reverse mode: the variants that keep the design window
    const bool wrec = adj_edge_mode(c);
    if (e == cudaSuccess && c->n_tasks_n > 0) {
        // whole-warp CPML tasks without the design in reach and the narrow x-slab
        // tasks, in one launch
        e = launch_cpml_mixed(c, sb, T, n0, parity);
        c->launches++;
    } else if (e == cudaSuccess && c->n_tasks_b > 0) {
        // CPML tasks with no design rectangle in reach: the build without design code
        e = launch_fused<7>(c->d_tasks_b, c->n_tasks_b, c->warps_b, c, sb, T, n0, parity);
        c->launches++;
    }
    if (e == cudaSuccess && c->n_tasks_bd > 0) {
        // CPML tasks with the design in reach follow on the same stream
        e = wrec ? launch_fused<5>(c->d_tasks_bd, c->n_tasks_bd, c->warps_b, c, sb, T, n0, parity)
                 : launch_fused<1>(c->d_tasks_bd, c->n_tasks_bd, c->warps_b, c, sb, T, n0, parity);
        c->launches++;
    }
    if (e == cudaSuccess && c->n_tasks_s > 0) {
        // split-field layer tasks follow the CPML ones on the same stream
        e = launch_fused<3>(c->d_tasks_s, c->n_tasks_s, c->warps_b, c, sb, T, n0, parity);
        c->launches++;
    }
    if (e == cudaSuccess && nl > 0) {
        e = wrec ? launch_fused<6>(c->d_tasks_l, nl, c->warps_l, c, sl, T, n0, parity)
                 : launch_fused<2>(c->d_tasks_l, nl, c->warps_l, c, sl, T, n0, parity);
        c->launches++;
    }
    if (e == cudaSuccess && ni > 0) {
        e = launch_fused<0>(c->d_tasks, ni, warps, c, c->stream, T, n0, parity);
        c->launches++;
    }
    if (e == cudaSuccess && sb != c->stream) {
        e = cudaEventRecord(c->ev_join, sb);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_join, 0);
    }
    if (e == cudaSuccess && sl != c->stream) {
        e = cudaEventRecord(c->ev_join2, sl);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_join2, 0);
    }
    if (e != cudaSuccess) {
        c->err = std::string("fused launch: ") + cudaGetErrorString(e);
        return FDTD_ECUDA;
    }
    return FDTD_OK;
}

int tmz_naive_step(fdtd_ctx* c, long long n) {
    int mx = 0, my = 0;
    for (auto* s : c->s2) {
        mx = s->nx > mx ? s->nx : mx;
        my = s->ny > my ? s->ny : my;
    }
    const dim3 blk(32, 8);
    const dim3 grd((mx + 31) / 32, (my + 7) / 8, (unsigned)c->s2.size());
    k_tmz_h<<<grd, blk, 0, c->stream>>>(c->d_scenes, c->parity);
    k_tmz_e<<<grd, blk, 0, c->stream>>>(c->d_scenes, c->parity);
    k_tmz_src_rec<<<(unsigned)c->s2.size(), 128, 0, c->stream>>>(c->d_scenes, c->d_samp_scene,
                                                                 c->d_samp_off, c->parity, n);
    c->launches += 3;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string("naive step: ") + cudaGetErrorString(e);
        return FDTD_ECUDA;
    }
    return FDTD_OK;
}

// effective (Ca, Cb/dx, Cb/dy) of every stored column of the design rows: the
// design value inside the rectangle, the material table's elsewhere
__global__ void k_design_band(const uint8_t* __restrict__ mat, const float4* __restrict__ coef,
                              const float4* __restrict__ dsg, float* __restrict__ band, int pitch, int i0, int j0,
                              int w, int h) {
    const int cs = blockIdx.x * blockDim.x + threadIdx.x;
    const int dj = blockIdx.y;
    if (cs >= pitch || dj >= h) return;
    const int i = cs - PAD_X;
    float4 co = coef[mat[(size_t)(j0 + dj + PAD_Y) * pitch + cs]];
    if (i >= i0 && i < i0 + w) co = dsg[(size_t)dj * w + (i - i0)];
    const size_t plane = (size_t)h * pitch, o = (size_t)dj * pitch + cs;
    band[o] = co.x;
    band[plane + o] = co.y;
    band[2 * plane + o] = co.z;
}

// eq. (7) for every design cell from device arrays (FP64, as the host path):
// co = (Ca, Cb/dx, Cb/dy, Cb) and the gradient factor -eps0 / (eps0 eps_r + sigma dt / 2);
// *bad = 1 if some eps_r <= 0 or sigma < 0 (or either is NaN)
__global__ void k_design_coeffs(const double* __restrict__ eps_r, const double* __restrict__ sigma, int n, double dt,
                                double dx, double dy, double eps0, float4* __restrict__ co, float* __restrict__ fac,
                                int* bad) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const double er = eps_r[q], sg = sigma ? sigma[q] : 0.0;
    if (!(er > 0.0) || !(sg >= 0.0)) {
        atomicOr(bad, 1);
        return;
    }
    const double eps = __dmul_rn(eps0, er);
    const double half = __ddiv_rn(__dmul_rn(sg, dt), __dmul_rn(2.0, eps));
    const double am = __dsub_rn(1.0, half), ap = __dadd_rn(1.0, half);
    const double ca = __ddiv_rn(am, ap), cb = __ddiv_rn(dt, __dmul_rn(ap, eps));
    co[q] = make_float4((float)ca, (float)__ddiv_rn(cb, dx), (float)__ddiv_rn(cb, dy), (float)cb);
    fac[q] = (float)__ddiv_rn(-eps0, __dadd_rn(eps, __ddiv_rn(__dmul_rn(sg, dt), 2.0)));
}

int tmz_design_coeffs(fdtd_ctx* c, Scene2* s, const double* eps_r, const double* sigma, size_t n, int* bad) {
    int* d_bad = nullptr;
    if (cudaMallocAsync(&d_bad, sizeof(int), c->stream) != cudaSuccess) return FDTD_ENOMEM;
    cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream);
    const double eps0 = 1.0 / (4.0e-7 * M_PI * 299792458.0 * 299792458.0);
    k_design_coeffs<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(eps_r, sigma, (int)n, s->dt, s->dx, s->dy,
                                                                         eps0, s->d_dsg, s->d_dsg_fac, d_bad);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(d_bad, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("design coefficients: ") + cudaGetErrorString(e);
        return FDTD_ECUDA;
    }
    return FDTD_OK;
}

int tmz_design_band(fdtd_ctx* c, Scene2* s) {
    const dim3 grd((unsigned)((s->pitch + 127) / 128), (unsigned)s->dsg_h);
    k_design_band<<<grd, 128, 0, c->stream>>>(s->d_mat, s->d_coef, s->d_dsg, s->d_band, s->pitch, s->dsg_i0,
                                             s->dsg_j0, s->dsg_w, s->dsg_h);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string("design band: ") + cudaGetErrorString(e);
        return FDTD_ECUDA;
    }
    return FDTD_OK;
}

// every cell-monitor accumulator of the context, one thread each, over the
// steps n0 .. n0 + nsteps - 1: F += E^{n+1} exp(-i 2 pi f (n+1) dt) dt.  The
// phase is exact in 64-bit fixed point; its sine and cosine are taken in FP32.
__global__ void k_dft_items(const DftItem* __restrict__ items, int n_items, long long n0, int nsteps) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n_items) return;
    const DftItem it = items[id];
    float4 a = *it.acc;
    for (int k = 0; k < nsteps; k++) {
        const long long n = n0 + k;
        const float e = it.rec[n * it.n_rec + it.slot];
        const unsigned long long ph = (unsigned long long)(n + 1) * it.inc;
        const float x = (float)(long long)ph * 5.42101086242752217e-20f;   // 2^-64: cycles in [-1/2, 1/2)
        float sn, cs;
        sincospif(2.f * x, &sn, &cs);
        kahan_add(a.x, a.z, e * (cs * it.dt));
        kahan_add(a.y, a.w, -e * (sn * it.dt));
    }
    *it.acc = a;
}

int dft_items_launch(fdtd_ctx* c, long long n0, int nsteps) {
    k_dft_items<<<(c->n_dft + 127) / 128, 128, 0, c->stream>>>(c->d_dft, c->n_dft, n0, nsteps);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string("dft: ") + cudaGetErrorString(e);
        return FDTD_ECUDA;
    }
    return FDTD_OK;
}

int dft_cells_launch(fdtd_ctx* c, const DftMon& m, long long n0, int nsteps) {
    const Scene2* s = c->s2[m.scene];
    const int n = m.n_cells * m.n_freq;
    k_dft_cells<<<(n + 127) / 128, 128, 0, c->stream>>>(s->d_rec, (int)s->samples.size(), m.slot0, m.n_cells,
                                                       m.d_freq, m.n_freq, s->dt, m.d_acc, n0, nsteps);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string("dft: ") + cudaGetErrorString(e);
        return FDTD_ECUDA;
    }
    return FDTD_OK;
}

// one scan of every scene's current Ez, Hx, Hy: sets *d_flag (device word) to 1
// if any value is not finite; never clears it
cudaError_t tmz_finite_launch(fdtd_ctx* c, int* d_flag) {
    int mx = 0, my = 0;
    for (auto* s : c->s2) {
        mx = s->nx > mx ? s->nx : mx;
        my = s->ny > my ? s->ny : my;
    }
    const dim3 blk(32, 8);
    const dim3 grd((mx + 31) / 32, (my + 7) / 8, (unsigned)c->s2.size());
    k_tmz_finite<<<grd, blk, 0, c->stream>>>(c->d_scenes, c->parity, d_flag);
    c->launches++;
    return cudaGetLastError();
}

int tmz_finite_check(fdtd_ctx* c, int* bad) {
    int* d_bad = nullptr;
    if (cudaMallocAsync(&d_bad, sizeof(int), c->stream) != cudaSuccess) return FDTD_ENOMEM;
    cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream);
    tmz_finite_launch(c, d_bad);
    cudaMemcpyAsync(bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(d_bad, c->stream);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("finite check: ") + cudaGetErrorString(e);
        return FDTD_ECUDA;
    }
    return FDTD_OK;
}

}  // namespace gem

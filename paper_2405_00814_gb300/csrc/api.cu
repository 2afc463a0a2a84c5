// Host side of the C ABI (include/gem_fdtd.h): contexts, inputs, coefficient
// tables, monitors and the step loop.  All arithmetic of the time step runs in
// the kernels; the host computes the per-material coefficients of eq. (7) and
// the CPML profiles once, in FP64, and rounds them to FP32.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <cstdint>
#include <string>
#include <vector>

#include "gem_internal.h"

using namespace gem;

namespace {

const double kC0 = 299792458.0;
const double kMu0 = 4.0e-7 * M_PI;
const double kEps0 = 1.0 / (kMu0 * kC0 * kC0);
// CPML grading (Roden & Gedney): polynomial order, alpha at the inner interface
const double kPmlM = 3.0;
const double kPmlAlphaMax = 0.05;

int fail(fdtd_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

int cuda_fail(fdtd_ctx* c, cudaError_t e, const char* what) {
    return fail(c, FDTD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                 \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

template <class P>
int dalloc(fdtd_ctx* c, P** p, size_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(c, FDTD_ENOMEM, "cudaMalloc %zu bytes for %s: %s", bytes, what, cudaGetErrorString(e));
    }
    return FDTD_OK;
}

void dfree(void* p) {
    if (p) cudaFree(p);
}

double courant_limit_2d(double dx, double dy) { return 1.0 / (kC0 * sqrt(1.0 / (dx * dx) + 1.0 / (dy * dy))); }

// one CPML point: depth rho (cells) from the inner interface of an npml-cell layer
void cpml_point(double rho, int npml, double delta, double dt, double* b, double* c) {
    if (rho <= 0.0 || npml <= 0) {
        *b = 0.0;
        *c = 0.0;
        return;
    }
    const double eta0 = sqrt(kMu0 / kEps0);
    const double smax = 0.8 * (kPmlM + 1.0) / (eta0 * delta);
    const double x = rho / npml;
    const double sig = smax * pow(x, kPmlM);
    const double alp = kPmlAlphaMax * (1.0 - x);
    const double bb = exp(-(sig + alp) * dt / kEps0);   // kappa = 1
    *b = bb;
    *c = sig * (bb - 1.0) / (sig + alp);
}

// profile arrays of one axis in storage coordinates: E nodes at integer
// positions, H nodes at +1/2; n cells, pad cells before index 0
void cpml_axis(int n, int npml, double delta, double dt, int pad, int len, float* bE, float* cE, float* bH,
               float* cH) {
    for (int k = 0; k < len; k++) bE[k] = cE[k] = bH[k] = cH[k] = 0.f;
    if (npml <= 0) return;
    for (int i = 0; i < n; i++) {
        const double xe = i, xh = i + 0.5, lo = npml, hi = n - npml;
        double rE = 0, rH = 0;
        if (xe < lo) rE = lo - xe;
        if (xe > hi) rE = xe - hi;
        if (xh < lo) rH = lo - xh;
        if (xh > hi) rH = xh - hi;
        double b, c;
        cpml_point(rE, npml, delta, dt, &b, &c);
        bE[i + pad] = (float)b;
        cE[i + pad] = (float)c;
        cpml_point(rH, npml, delta, dt, &b, &c);
        bH[i + pad] = (float)b;
        cH[i + pad] = (float)c;
    }
}

// Berenger split-field layer (Sec. III-C): conductivity sigma_max (depth/d)^3,
// sigma_max = 0.8 (m+1) / (eta0 delta) with m = 3, E nodes at integer and H nodes
// at half-integer depth.  Per node of one axis, in storage coordinates:
// Ca, Cb/delta of the E part along this axis (vacuum, eq. (7) with sigma) and
// Da, Db/delta of the H component damped by this axis (sigma* = sigma mu0/eps0).
// Nodes outside the layer hold the vacuum values (sigma = 0).
void split_axis(int n, int npml, double delta, double dt, int pad, int len, float* caE, float* cbE, float* daH,
                float* dbH) {
    for (int k = 0; k < len; k++) caE[k] = cbE[k] = daH[k] = dbH[k] = 0.f;
    const double eta0 = sqrt(kMu0 / kEps0);
    const double smax = 0.8 * (kPmlM + 1.0) / (eta0 * delta);
    for (int i = 0; i < n; i++) {
        const double xe = i, xh = i + 0.5, lo = npml, hi = n - npml;
        double rE = 0, rH = 0;
        if (xe < lo) rE = lo - xe;
        if (xe > hi) rE = xe - hi;
        if (xh < lo) rH = lo - xh;
        if (xh > hi) rH = xh - hi;
        const double sE = smax * pow(rE / npml, kPmlM), sH = smax * pow(rH / npml, kPmlM);
        const double ae = 1.0 + sE * dt / (2.0 * kEps0);
        caE[i + pad] = (float)((1.0 - sE * dt / (2.0 * kEps0)) / ae);
        cbE[i + pad] = (float)(dt / (kEps0 * ae) / delta);
        const double ah = 1.0 + sH * dt / (2.0 * kEps0);   // sigma* dt / (2 mu0) = sigma dt / (2 eps0)
        daH[i + pad] = (float)((1.0 - sH * dt / (2.0 * kEps0)) / ah);
        dbH[i + pad] = (float)(dt / (kMu0 * ah) / delta);
    }
}

// an E node of the split layer (positive depth on either axis)
bool split_layer_cell(int i, int j, int nx, int ny, int npml) {
    return i < npml || i > nx - npml || j < npml || j > ny - npml;
}

// eq. (7): Ca = A_-/A_+, Cb = dt/(A_+ eps), A_-/+ = 1 -/+ sigma dt/(2 eps)
float4 e_coeffs(double eps_r, double sigma, double dt, double dx, double dy) {
    const double eps = kEps0 * eps_r;
    const double am = 1.0 - sigma * dt / (2.0 * eps);
    const double ap = 1.0 + sigma * dt / (2.0 * eps);
    const double ca = am / ap, cb = dt / (ap * eps);
    return make_float4((float)ca, (float)(cb / dx), (float)(cb / dy), (float)cb);
}

double waveform(int kind, double p, double t) {
    if (kind == FDTD_SRC_RICKER) {
        const double tau = t - 1.5 / p;
        const double a = M_PI * M_PI * p * p * tau * tau;
        return (1.0 - 2.0 * a) * exp(-a);
    }
    const double tg = 1.0 / p, t0 = 4.0 * tg, u = (t - t0) / tg;
    if (kind == FDTD_SRC_GAUSS_MOD) return exp(-u * u) * sin(2.0 * M_PI * p * (t - t0));
    if (kind == FDTD_SRC_GAUSS) return exp(-u * u);
    if (kind == FDTD_SRC_SINE) return sin(2.0 * M_PI * p * t);
    return 0.0;
}

Scene2* cur2(fdtd_ctx* c) { return (c->dims == 2 && !c->s2.empty()) ? c->s2[c->cur] : nullptr; }

void scene2_free(Scene2* s) {
    if (!s) return;
    for (int f = 0; f < F_COUNT2; f++)
        for (int p = 0; p < 2; p++) dfree(s->fbuf[f][p]);
    dfree(s->d_mat);
    dfree(s->d_coef);
    dfree(s->d_prof);
    dfree(s->d_src);
    dfree(s->d_rec);
    dfree(s->d_dsg);
    dfree(s->d_band);
    dfree(s->d_dsg_fac);
    delete s;
}

// the PEC walls i = 0 and j = 0 of a padded material map take PEC_MAT (row 0
// only when it is the wall: a slab above the grid's first row has none)
__global__ void k_pec_walls(uint8_t* __restrict__ mat, int pitch, int nx, int ny, int wall_row0) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < nx) {
        if (wall_row0) mat[(size_t)PAD_Y * pitch + PAD_X + q] = (uint8_t)PEC_MAT;
    } else if (q < nx + ny) {
        mat[(size_t)(q - nx + PAD_Y) * pitch + PAD_X] = (uint8_t)PEC_MAT;
    }
}

static int pec_walls(fdtd_ctx* c, Scene2* s) {
    const int n = s->nx + s->ny;
    k_pec_walls<<<(n + 255) / 256, 256, 0, c->stream>>>(s->d_mat, s->pitch, s->nx, s->ny, s->yoff == 0 ? 1 : 0);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "PEC walls");
    return FDTD_OK;
}

// owned rows [j0, j1) of a y-slab sub-domain and its halo depth
struct SlabSpec {
    int j0, j1, ghost;
};

int scene2_init(fdtd_ctx* c, const fdtd_grid* g, double dx, double dt, double courant, const uint8_t* mat,
                const fdtd_material* table, int n_mat, Scene2** out, const SlabSpec* slab = nullptr) {
    *out = nullptr;
    if (!g || !mat || !table) return fail(c, FDTD_EINVAL, "NULL grid, material map or table");
    if (g->dims != 2) return fail(c, FDTD_EINVAL, "scene dims %d: this entry handles 2D", g->dims);
    if (g->nx < 4 || g->ny < 4) return fail(c, FDTD_EINVAL, "grid %dx%d too small (>= 4 cells per axis)", g->nx, g->ny);
    // a slab holds rows [j0 - ghost_lo, j1 + ghost_hi) of the grid
    int yoff = 0, ny_loc = g->ny, ghost = 0, ghost_lo = 0, ghost_hi = 0;
    if (slab) {
        ghost = slab->ghost;
        if (ghost < 1 || ghost > 64) return fail(c, FDTD_EINVAL, "ghost depth %d outside 1..64", ghost);
        if (slab->j0 < 0 || slab->j1 > g->ny || slab->j1 - slab->j0 < ghost)
            return fail(c, FDTD_EINVAL, "slab rows [%d, %d) of %d: need 0 <= j0, j1 <= ny and at least %d owned rows",
                        slab->j0, slab->j1, g->ny, ghost);
        ghost_lo = slab->j0 > 0 ? ghost : 0;
        ghost_hi = slab->j1 < g->ny ? ghost : 0;
        if (slab->j0 - ghost_lo < 0 || slab->j1 + ghost_hi > g->ny)
            return fail(c, FDTD_EINVAL, "slab [%d, %d): its %d ghost rows leave the grid", slab->j0, slab->j1, ghost);
        if (g->boundary == FDTD_SPLIT_PML) return fail(c, FDTD_EINVAL, "slab sub-domains cover PEC and CPML grids");
        yoff = slab->j0 - ghost_lo;
        ny_loc = slab->j1 - slab->j0 + ghost_lo + ghost_hi;
        if (ny_loc < 4) return fail(c, FDTD_EINVAL, "slab of %d rows too small (>= 4)", ny_loc);
    }
    if ((int64_t)g->nx * g->ny > (int64_t)1 << 31) return fail(c, FDTD_EINVAL, "grid too large");
    if (!(dx > 0)) return fail(c, FDTD_EINVAL, "dx must be > 0");
    const double dy = g->dy > 0 ? g->dy : dx;
    int npml = 0;
    const bool split = g->boundary == FDTD_SPLIT_PML;
    if (g->boundary == FDTD_CPML || split) {
        npml = g->pml_cells;
        if (npml < 1 || 2 * npml + 2 > std::min(g->nx, g->ny))
            return fail(c, FDTD_EINVAL, "pml_cells %d does not fit a %dx%d grid", npml, g->nx, g->ny);
    } else if (g->boundary != FDTD_PEC) {
        return fail(c, FDTD_EINVAL, "unknown boundary %d", g->boundary);
    }
    const double lim = courant_limit_2d(dx, dy);
    if (dt <= 0) {
        if (!(courant > 0 && courant <= 1.0)) return fail(c, FDTD_EINVAL, "courant factor must be in (0, 1]");
        dt = courant * lim;
    } else if (dt > lim) {
        return fail(c, FDTD_EUNSTABLE, "dt %.6g s exceeds the 2D Courant limit %.6g s", dt, lim);
    }
    if (n_mat < 1 || n_mat > 255) return fail(c, FDTD_EINVAL, "n_mat %d outside 1..255", n_mat);
    for (int m = 0; m < n_mat; m++) {
        if (!(table[m].eps_r > 0)) return fail(c, FDTD_EINVAL, "material %d: eps_r must be > 0", m);
        if (table[m].mu_r != 1.0) return fail(c, FDTD_EINVAL, "material %d: mu_r must be 1 (non-magnetic medium)", m);
        if (!(table[m].sigma >= 0)) return fail(c, FDTD_EINVAL, "material %d: sigma must be >= 0", m);
    }
    const int64_t ncell = (int64_t)g->nx * ny_loc;
    {
        uint8_t mx = 0;   // a branch-free pass first; the offending cell is looked up only on failure
        for (int64_t k = 0; k < ncell; k++) mx = mat[k] > mx ? mat[k] : mx;
        if (mx >= n_mat)
            for (int64_t k = 0; k < ncell; k++)
                if (mat[k] >= n_mat)
                    return fail(c, FDTD_EINVAL, "material index %d at cell %lld >= n_mat %d", mat[k], (long long)k, n_mat);
    }
    if (split) {
        // the split layer's coefficients are per-axis profiles of vacuum
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                if (!split_layer_cell(i, j, g->nx, g->ny, npml)) continue;
                const int m = mat[(size_t)j * g->nx + i];
                if (table[m].eps_r != 1.0 || table[m].sigma != 0.0)
                    return fail(c, FDTD_EINVAL, "split-field PML: cell (%d, %d) in the layer is not vacuum", i, j);
            }
    }

    Scene2* s = new Scene2();
    memset((void*)s->fbuf, 0, sizeof(s->fbuf));
    s->d_mat = nullptr; s->d_coef = nullptr; s->d_prof = nullptr; s->d_src = nullptr; s->d_rec = nullptr;
    s->d_dsg = nullptr;
    s->d_band = nullptr;
    s->d_dsg_fac = nullptr;
    s->nx = g->nx; s->ny = ny_loc; s->npml = npml; s->split = split ? 1 : 0;
    s->yoff = yoff; s->ny_glob = g->ny; s->ghost = ghost; s->ghost_lo = ghost_lo; s->ghost_hi = ghost_hi;
    s->dx = dx; s->dy = dy; s->dt = dt;
    s->pitch = ((PAD_X + g->nx + STRIP) + 31) / 32 * 32;
    s->rows = ny_loc + 2 * PAD_Y;
    s->eps_r.resize(n_mat);
    s->sigma.resize(n_mat);
    for (int m = 0; m < n_mat; m++) {
        s->eps_r[m] = table[m].eps_r;
        s->sigma[m] = table[m].sigma;
    }
    s->src_kind = -1; s->src_i = -1; s->src_j = -1; s->src_j1 = -1; s->src_param = 0; s->src_cap = 0;
    s->rec_cap = 0;
    s->dsg_i0 = s->dsg_j0 = s->dsg_w = s->dsg_h = 0;

    const size_t fbytes = (size_t)s->pitch * s->rows * sizeof(float);
    for (int f = 0; f < F_COUNT2; f++)
        for (int p = 0; p < 2; p++) {
            int rc = dalloc(c, &s->fbuf[f][p], fbytes, "field");
            if (rc) { scene2_free(s); return rc; }
            cudaMemsetAsync(s->fbuf[f][p], 0, fbytes, c->stream);
        }
    // padded material map: pads and the PEC walls i = 0, j = 0 get PEC_MAT (the
    // map is copied into the padded layout on the device, walls marked after)
    const size_t mat_bytes = (size_t)s->pitch * s->rows;
    int rc = dalloc(c, &s->d_mat, mat_bytes, "material map");
    if (rc) { scene2_free(s); return rc; }
    // coefficient table
    std::vector<float4> co(256, make_float4(0, 0, 0, 0));
    for (int m = 0; m < n_mat; m++) co[m] = e_coeffs(table[m].eps_r, table[m].sigma, dt, dx, dy);
    rc = dalloc(c, &s->d_coef, 256 * sizeof(float4), "coefficients");
    if (rc) { scene2_free(s); return rc; }
    // CPML profiles
    std::vector<float> prof(4 * (size_t)s->pitch + 4 * (size_t)s->rows, 0.f);
    float* px = prof.data();
    float* py = prof.data() + 4 * s->pitch;
    if (split) {
        split_axis(s->nx, npml, dx, dt, PAD_X, s->pitch, px, px + s->pitch, px + 2 * s->pitch, px + 3 * s->pitch);
        split_axis(s->ny, npml, dy, dt, PAD_Y, s->rows, py, py + s->rows, py + 2 * s->rows, py + 3 * s->rows);
    } else {
        cpml_axis(s->nx, npml, dx, dt, PAD_X, s->pitch, px, px + s->pitch, px + 2 * s->pitch, px + 3 * s->pitch);
        // y: the whole grid's profile, then the slab's window of it
        const int rows_g = g->ny + 2 * PAD_Y;
        std::vector<float> pg(4 * (size_t)rows_g);
        cpml_axis(g->ny, npml, dy, dt, PAD_Y, rows_g, pg.data(), pg.data() + rows_g, pg.data() + 2 * rows_g,
                  pg.data() + 3 * rows_g);
        for (int q = 0; q < 4; q++)
            for (int r = 0; r < s->rows; r++) py[(size_t)q * s->rows + r] = pg[(size_t)q * rows_g + r + yoff];
    }
    rc = dalloc(c, &s->d_prof, prof.size() * sizeof(float), "profiles");
    if (rc) { scene2_free(s); return rc; }
    cudaError_t e = cudaMemsetAsync(s->d_mat, PEC_MAT, mat_bytes, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(s->d_mat + (size_t)PAD_Y * s->pitch + PAD_X, s->pitch, mat, s->nx, s->nx, s->ny,
                              cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && pec_walls(c, s) != FDTD_OK) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_coef, co.data(), 256 * sizeof(float4), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_prof, prof.data(), prof.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) { scene2_free(s); return cuda_fail(c, e, "upload scene"); }
    *out = s;
    return FDTD_OK;
}

fdtd_ctx* ctx_new(void* stream) {
    fdtd_ctx* c = new fdtd_ctx();
    c->dims = 2;
    c->stream = (cudaStream_t)stream;
    c->s3 = nullptr;
    c->cur = 0;
    c->t = 0;
    c->parity = 0;
    c->launches = 0;
    c->opt_kernel = 0;
    c->opt_tblock = 4;
    c->opt_warps = 8;
    c->opt_segment = 64;
    c->opt_segment_b = 0;
    c->opt_taper = 0;
    c->opt_warps_b = 2;
    c->opt_playout = 0;
    c->opt_bulk = 0;
    c->use_bulk = 0;
    c->d_bulk_err = nullptr;
    c->task_warps_b = 0;
    c->dirty = true;
    c->d_scenes = nullptr;
    c->d_tasks = nullptr;
    c->d_tasks_b = nullptr;
    c->n_tasks_b = 0;
    c->warps_b = 2;
    c->d_tasks_l = nullptr;
    c->n_tasks_l = 0;
    c->warps_l = 4;
    c->d_tasks_s = nullptr;
    c->n_tasks_s = 0;
    c->d_tasks_bd = nullptr;
    c->n_tasks_bd = 0;
    c->d_tasks_n = nullptr;
    c->n_tasks_n = 0;
    c->task_narrow = -1;
    c->task_pers = -1;
    c->aux = c->aux2 = nullptr;
    c->ev_fork = c->ev_join = c->ev_join2 = nullptr;
    cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&c->aux2, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming);
    c->d_samp = nullptr;
    c->d_samp_scene = nullptr;
    c->d_samp_off = nullptr;
    c->n_tasks = 0;
    c->task_tb = c->task_seg = -1;
    c->graph = nullptr;
    c->adj = nullptr;
    c->d_ptasks = nullptr; c->d_pitems = nullptr; c->d_dep_off = nullptr; c->d_dep_idx = nullptr; c->d_done = nullptr;
    c->d_dft = nullptr;
    c->n_dft = 0;
    c->n_pitems = 0;
    c->d_ctl = nullptr;
    c->ctl_words = 0;
    c->h_err = nullptr;
    if (cudaMallocHost(&c->h_err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        c->h_err = nullptr;
    } else {
        *c->h_err = 0;
    }
    c->spin_limit = 4000000;   // about half a second of polls
    c->opt_debug_skip = -1;
    c->opt_adj_store = 1;
    c->opt_check_every = 0;
    c->d_bad = nullptr;
    c->h_bad = nullptr;
    if (cudaMallocHost(&c->h_bad, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        c->h_bad = nullptr;
    } else {
        *c->h_bad = 0;
    }
    c->opt_graph = 0;
    c->graph_exec = nullptr;
    c->graph_t = c->graph_n = -1;
    c->graph_parity = 0;
    c->cap_stream = nullptr;
    return c;
}

// source waveform and sample record must cover steps [0, t_end)
int ensure_capacity(fdtd_ctx* c, int64_t t_end) {
    for (Scene2* s : c->s2) {
        if (s->src_kind >= 0 && s->src_cap < t_end) {
            int64_t cap = std::max<int64_t>(t_end, 2 * s->src_cap);
            cap = std::max<int64_t>(cap, 1024);
            std::vector<float> w((size_t)cap, 0.f);
            for (int64_t n = 0; n < cap; n++) {
                if (s->src_kind == FDTD_SRC_SAMPLED)
                    w[n] = n < (int64_t)s->src_samples.size() ? s->src_samples[n] : 0.f;
                else
                    w[n] = (float)waveform(s->src_kind, s->src_param, (double)(n + 1) * s->dt);
            }
            float* d = nullptr;
            int rc = dalloc(c, &d, (size_t)cap * sizeof(float), "source waveform");
            if (rc) return rc;
            CK(cudaMemcpyAsync(d, w.data(), (size_t)cap * sizeof(float), cudaMemcpyHostToDevice, c->stream), "upload waveform");
            CK(cudaStreamSynchronize(c->stream), "upload waveform");
            dfree(s->d_src);
            s->d_src = d;
            s->src_cap = cap;
            c->dirty = true;
        }
        const int nrec = (int)s->samples.size();
        if (nrec > 0 && s->rec_cap < t_end) {
            int64_t cap = std::max<int64_t>(t_end, 2 * s->rec_cap);
            cap = std::max<int64_t>(cap, 1024);
            float* d = nullptr;
            const size_t bytes = (size_t)cap * nrec * sizeof(float);
            int rc = dalloc(c, &d, bytes, "sample record");
            if (rc) return rc;
            CK(cudaMemsetAsync(d, 0, bytes, c->stream), "record memset");
            if (s->d_rec && s->rec_cap > 0)
                CK(cudaMemcpyAsync(d, s->d_rec, (size_t)s->rec_cap * nrec * sizeof(float), cudaMemcpyDeviceToDevice,
                                   c->stream), "record copy");
            CK(cudaStreamSynchronize(c->stream), "record grow");
            dfree(s->d_rec);
            s->d_rec = d;
            s->rec_cap = cap;
            c->dirty = true;
        }
    }
    return FDTD_OK;
}

// device scene descriptors, fused-kernel task list and sample lists
int rebuild(fdtd_ctx* c, int T, int seg, int warps) {
    // a recorded graph holds the buffers about to be replaced
    if (c->graph_exec) {
        cudaGraphExecDestroy((cudaGraphExec_t)c->graph_exec);
        c->graph_exec = nullptr;
        c->graph_t = c->graph_n = -1;
    }
    const int ns = (int)c->s2.size();
    std::vector<TmzDev> dev(ns);
    for (int k = 0; k < ns; k++) {
        Scene2* s = c->s2[k];
        TmzDev& d = dev[k];
        memset(&d, 0, sizeof(d));
        for (int f = 0; f < F_COUNT2; f++)
            for (int p = 0; p < 2; p++) d.f[f][p] = s->fbuf[f][p];
        d.mat = s->d_mat;
        d.coef = s->d_coef;
        d.prof = s->d_prof;
        d.nx = s->nx; d.ny = s->ny; d.pitch = s->pitch; d.rows = s->rows;
        d.has_pml = s->split ? 0 : s->npml;
        d.split = s->split ? s->npml : 0;
        d.dbx = (float)(s->dt / (kMu0 * s->dx));
        d.dby = (float)(s->dt / (kMu0 * s->dy));
        d.src_i = s->src_kind >= 0 ? s->src_i : -1;
        d.src_j = s->src_kind >= 0 ? s->src_j : -1;
        d.src_j1 = s->src_kind >= 0 ? s->src_j1 : -1;
        d.src_wave = s->d_src;
        d.src_len = s->src_kind >= 0 ? s->src_cap : 0;
        d.rec = s->d_rec;
        d.n_rec = (int)s->samples.size();
        d.rec_cap = s->rec_cap;
        d.dsg_i0 = s->dsg_i0; d.dsg_j0 = s->dsg_j0; d.dsg_w = s->d_dsg ? s->dsg_w : 0; d.dsg_h = s->dsg_h;
        d.dsg_coef = s->d_dsg;
        d.dsg_band = s->d_band;
        d.pml_ylo = s->npml - s->yoff;
        d.pml_yhi = s->ny_glob - s->npml - s->yoff;
    }
    // tasks: per scene, strips of 120 columns x segments of seg rows.  Tasks
    // with a CPML slab or the design rectangle within reach go to the boundary
    // list, the rest to the interior list; each list is padded to whole CTAs
    // per scene so that a CTA never mixes scenes.
    const int wout = STRIP - 2 * HALO;
    std::vector<Task> tasks, tasks_b, tasks_l, tasks_s, tasks_bd, tasks_n;
    std::vector<Sample2> tsamp;
    const int warps_b = c->opt_warps_b;
    const bool want_narrow = c->opt_kernel == 0 || c->opt_kernel == 2;   // not the unfused pair
    bool any_design = false;
    for (const Scene2* s : c->s2) any_design = any_design || s->d_dsg != nullptr;
    const int warps_l = 4;   // lite CTAs; each list is padded to its launch's CTA width
    for (int k = 0; k < ns; k++) {
        Scene2* s = c->s2[k];
        const size_t first = tasks.size(), first_b = tasks_b.size(), first_l = tasks_l.size(),
                     first_s = tasks_s.size(), first_bd = tasks_bd.size();
        // Tasks with a CPML slab, the design rectangle, the source or a probe in
        // reach, or a ragged right edge, run the general kernel ("boundary" list);
        // the rest run the lean interior kernel.  General warps are heavier per
        // row, so they get half-height segments.
        const int seg_b = c->opt_segment_b > 0 ? c->opt_segment_b : std::max(8, seg / 2);
        // Narrow x-slab tasks: the columns [0, NG_OWN) and [xr, nx) holding the
        // x-slabs of a CPML go to lane-group tasks (4 per warp) instead of whole
        // 120-column strips, and the strips cover [NG_OWN, xr) with a column
        // limit.  A strip computes the slab cells in its reach without the CPML,
        // which spoils one more column per step: its owned columns end at
        // xr <= nx - npml - MAX_TB, and its first loaded column NG_OWN - HALO is
        // outside the left slab.  The design rectangle must stay clear of the
        // narrow columns (those tasks are built without design code).
        const int xr = (s->nx - NG_OWN + 3) / 4 * 4;
        const bool nar = want_narrow && s->npml > 0 && !s->split && s->nx >= 2 * NG_OWN + 8 &&
                         NG_OWN - HALO >= s->npml && xr <= s->nx - s->npml - MAX_TB &&
                         !(s->d_dsg && (s->dsg_i0 < NG_OWN + HALO || s->dsg_i0 + s->dsg_w > xr - HALO));
        const int xl = nar ? NG_OWN : 0;
        auto owned_end = [&](int x0) { return nar ? std::min(x0 + wout, xr) : x0 + wout; };
        auto flags_of = [&](int x0, int ya, int yb, bool* general) {
            int f = 0;
            const int lx0 = x0 - HALO, lx1 = x0 - HALO + STRIP;   // loaded columns
            const int ly0 = ya - MAX_TB, ly1 = yb + MAX_TB;        // widest streamed rows
            const bool xslab = !nar && (lx0 < s->npml || lx1 > s->nx - s->npml);
            if (s->npml > 0 && (xslab || ly0 < s->npml - s->yoff || ly1 > s->ny_glob - s->npml - s->yoff))
                f |= TASK_PML;
            if (s->src_kind >= 0 && s->src_i >= lx0 && s->src_i < lx1 && s->src_j < ly1 && s->src_j1 > ly0)
                f |= TASK_SRC;
            if (s->d_dsg && s->dsg_i0 < lx1 && s->dsg_i0 + s->dsg_w > lx0 && s->dsg_j0 < ly1 && s->dsg_j0 + s->dsg_h > ly0)
                f |= TASK_DSG;
            bool samp = false;
            for (const Sample2& sp : s->samples)
                if (sp.i >= x0 && sp.i < owned_end(x0) && sp.j >= ya && sp.j < yb) samp = true;
            *general = f != 0 || samp || (!nar && x0 + wout > s->nx);
            return f;
        };
        auto add_task = [&](int x0, int ya, int yb) {
            Task t;
            bool general;
            t.scene = k; t.x0 = x0; t.ya = ya; t.yb = yb; t.xe = nar ? owned_end(x0) : 0;
            t.flags = flags_of(x0, ya, yb, &general);
            t.samp_begin = (int)tsamp.size();
            for (const Sample2& sp : s->samples)
                if (sp.i >= x0 && sp.i < owned_end(x0) && sp.j >= ya && sp.j < yb) tsamp.push_back(sp);
            t.samp_end = (int)tsamp.size();
            // the lite kernel pays for its own launch and stream fork only when a
            // design rectangle gives it work; otherwise its tasks join the CPML list
            // tasks within reach of a split-field layer run the split variant
            // CPML tasks with the design in reach run the build with design code,
            // all other CPML tasks the design-free one
            if ((t.flags & TASK_PML) && s->split) tasks_s.push_back(t);
            else if ((t.flags & TASK_PML) && (t.flags & TASK_DSG)) tasks_bd.push_back(t);
            else if ((t.flags & TASK_PML) || (general && !any_design)) tasks_b.push_back(t);
            else if (general) tasks_l.push_back(t);
            else tasks.push_back(t);
        };
        // the narrow tasks: both sides, segments of seg_b rows, the first task of
        // each warp repeated (TASK_NOSTORE) to fill the warp's four lane groups
        const size_t first_n = tasks_n.size();
        if (nar) {
            for (int side = 0; side < 2; side++) {
                const int x0 = side == 0 ? 0 : xr, xe = side == 0 ? NG_OWN : s->nx;
                for (int y = 0; y < s->ny; y += seg_b) {
                    Task t;
                    t.scene = k; t.x0 = x0; t.ya = y; t.yb = std::min(y + seg_b, s->ny); t.xe = xe;
                    t.flags = TASK_PML;
                    const int ly0 = t.ya - MAX_TB, ly1 = t.yb + MAX_TB;
                    if (s->src_kind >= 0 && s->src_i >= x0 - HALO && s->src_i < x0 - HALO + 4 * NG_LANES &&
                        s->src_j < ly1 && s->src_j1 > ly0)
                        t.flags |= TASK_SRC;
                    t.samp_begin = (int)tsamp.size();
                    for (const Sample2& sp : s->samples)
                        if (sp.i >= x0 && sp.i < xe && sp.j >= t.ya && sp.j < t.yb) tsamp.push_back(sp);
                    t.samp_end = (int)tsamp.size();
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
        // row segments: the rows within reach of a y-slab of the CPML, [0, y_lo)
        // and [y_hi, ny), in boundary-task heights, the rows between in
        // segments of seg rows, so that no segment reaches a slab by a few rows
        std::vector<std::pair<int, int>> segs;
        {
            int y_lo = 0, y_hi = s->ny;
            if (s->npml > 0) {
                y_lo = std::min(s->ny, std::max(0, s->npml - s->yoff + MAX_TB));
                y_hi = std::max(y_lo, std::min(s->ny, s->ny_glob - s->npml - s->yoff - MAX_TB));
            }
            // FDTD_OPT_TAPER (kernel 0): the last taper % of the rows between in
            // half-height tail segments, which the interior list runs last
            const int y_tail = c->opt_kernel == 0 && c->opt_taper > 0
                                   ? y_hi - (y_hi - y_lo) * c->opt_taper / 100 / 4 * 4 : y_hi;
            const int seg_t = std::max(8, seg / 2 / 4 * 4);
            for (int y = 0; y < y_lo; y += seg_b) segs.emplace_back(y, std::min(y + seg_b, y_lo));
            for (int y = y_lo; y < y_tail; y += seg) segs.emplace_back(y, std::min(y + seg, y_tail));
            for (int y = y_tail; y < y_hi; y += seg_t) segs.emplace_back(y, std::min(y + seg_t, y_hi));
            for (int y = y_hi; y < s->ny; y += seg_b) segs.emplace_back(y, std::min(y + seg_b, s->ny));
        }
        for (const auto& sg : segs) {
            const int ya = sg.first, yb = sg.second;
            for (int x0 = xl; x0 < (nar ? xr : s->nx); x0 += wout) {
                bool general;
                flags_of(x0, ya, yb, &general);
                if (!general) {
                    add_task(x0, ya, yb);
                } else {
                    for (int y = ya; y < yb; y += seg_b) add_task(x0, y, std::min(y + seg_b, yb));
                }
            }
        }
        Task pad;
        memset(&pad, 0, sizeof(pad));
        pad.scene = -1;
        if (tasks.size() > first)
            while ((tasks.size() - first) % warps) tasks.push_back(pad);
        if (tasks_b.size() > first_b)
            while ((tasks_b.size() - first_b) % warps_b) tasks_b.push_back(pad);
        if (tasks_l.size() > first_l)
            while ((tasks_l.size() - first_l) % warps_l) tasks_l.push_back(pad);
        if (tasks_s.size() > first_s)
            while ((tasks_s.size() - first_s) % warps_b) tasks_s.push_back(pad);
        if (tasks_bd.size() > first_bd)
            while ((tasks_bd.size() - first_bd) % warps_b) tasks_bd.push_back(pad);
        if (tasks_n.size() > first_n)   // whole CTAs of warps_b warps; a padding warp returns
            while ((tasks_n.size() - first_n) % (warps_b * 32 / NG_LANES)) tasks_n.push_back(pad);
    }
    // FDTD_OPT_TAPER: the interior list's CTAs (whole blocks of one scene each)
    // tallest first, in space order among equals
    if (c->opt_kernel == 0 && c->opt_taper > 0 && !tasks.empty()) {
        const size_t nb = tasks.size() / (size_t)warps;
        std::vector<std::pair<int, size_t>> key(nb);
        for (size_t b = 0; b < nb; b++) {
            int h = 0;
            for (int q = 0; q < warps; q++) {
                const Task& t = tasks[b * warps + q];
                if (t.scene >= 0) h = std::max(h, t.yb - t.ya);
            }
            key[b] = {-h, b};
        }
        std::stable_sort(key.begin(), key.end());
        std::vector<Task> sorted;
        sorted.reserve(tasks.size());
        for (const auto& kb : key)
            sorted.insert(sorted.end(), tasks.begin() + kb.second * warps, tasks.begin() + (kb.second + 1) * warps);
        tasks.swap(sorted);
    }
    // every list is launched in blocks of its own width: a block holds tasks of one
    // scene and starts with a real task, and every task lies inside its scene
    auto valid = [&](const std::vector<Task>& L, int width, const char* what) {
        if (L.size() % width) return fail(c, FDTD_ESTATE, "internal: %s list not padded to %d", what, width);
        for (size_t b = 0; b < L.size(); b += width) {
            const int sc = L[b].scene;
            if (sc < 0 || sc >= ns) return fail(c, FDTD_ESTATE, "internal: %s block %zu starts with padding", what, b);
            for (int q = 0; q < width; q++) {
                const Task& t = L[b + q];
                if (t.scene < 0) continue;
                const Scene2* s = c->s2[t.scene];
                if (t.scene != sc || t.x0 < 0 || t.x0 >= s->nx || t.ya < 0 || t.ya >= t.yb || t.yb > s->ny)
                    return fail(c, FDTD_ESTATE, "internal: %s task %zu out of its scene", what, b + q);
            }
        }
        return (int)FDTD_OK;
    };
    {
        int vr = valid(tasks, warps, "interior");
        if (!vr) vr = valid(tasks_b, warps_b, "CPML");
        if (!vr) vr = valid(tasks_bd, warps_b, "CPML design");
        if (!vr) vr = valid(tasks_s, warps_b, "split");
        if (!vr) vr = valid(tasks_l, warps_l, "lite");
        if (!vr) vr = valid(tasks_n, warps_b * 32 / NG_LANES, "narrow CPML");
        if (vr) return vr;
    }
    std::vector<Sample2> ssamp;
    std::vector<int> soff(ns + 1, 0);
    for (int k = 0; k < ns; k++) {
        for (const Sample2& sp : c->s2[k]->samples) ssamp.push_back(sp);
        soff[k + 1] = (int)ssamp.size();
    }
    // the persistent kernel's items, in space order (scene, strip, row): an item
    // of block b then waits for items of block b - 1 that were claimed about one
    // block's worth of work earlier, so blocks overlap instead of draining; each
    // item waits for the items of the previous block whose regions meet its own
    std::vector<Task> ptasks;
    std::vector<int2> pitems;
    const int per_warp_n = 32 / NG_LANES;
    if (c->opt_kernel == 2) {
        struct It { int kind; std::vector<Task> t; };
        std::vector<It> its;
        for (size_t q = 0; q + per_warp_n <= tasks_n.size(); q += per_warp_n) {
            if (tasks_n[q].scene < 0) continue;
            its.push_back({PITEM_NARROW, std::vector<Task>(tasks_n.begin() + q, tasks_n.begin() + q + per_warp_n)});
        }
        for (const std::vector<Task>* L : {&tasks_b, &tasks_bd, &tasks_l, &tasks})
            for (const Task& t : *L)
                if (t.scene >= 0) its.push_back({L == &tasks ? PITEM_INTERIOR : PITEM_GENERAL, {t}});
        std::stable_sort(its.begin(), its.end(), [](const It& a, const It& b) {
            const Task &p = a.t[0], &q = b.t[0];
            if (p.scene != q.scene) return p.scene < q.scene;
            if (p.x0 != q.x0) return p.x0 < q.x0;
            return p.ya < q.ya;
        });
        for (const It& it : its) {
            pitems.push_back(make_int2(it.kind, (int)ptasks.size()));
            ptasks.insert(ptasks.end(), it.t.begin(), it.t.end());
        }
    }
    std::vector<int> dep_off(pitems.size() + 1, 0), dep_idx;
    {
        // a task reads columns [x0 - HALO, x0 - HALO + 4 lanes) and rows
        // [ya - MAX_TB, yb + MAX_TB); it owns [x0, xe) x [ya, yb) (nothing for a
        // lane-group filler copy).  Two items depend on each other when one's
        // read box meets the other's owned box.
        struct Box { int scene, item, rx0, rx1, ry0, ry1, ox0, ox1, oy0, oy1; };
        std::vector<Box> bx;
        for (size_t i = 0; i < pitems.size(); i++) {
            const int n = pitems[i].x == PITEM_NARROW ? per_warp_n : 1;
            const int lanes = pitems[i].x == PITEM_NARROW ? NG_LANES : 32;
            for (int g = 0; g < n; g++) {
                const Task& t = ptasks[(size_t)pitems[i].y + g];
                const Scene2* s = c->s2[t.scene];
                Box b;
                b.scene = t.scene; b.item = (int)i;
                b.rx0 = t.x0 - HALO; b.rx1 = t.x0 - HALO + 4 * lanes;
                b.ry0 = t.ya - MAX_TB; b.ry1 = t.yb + MAX_TB;
                b.ox0 = t.x0;
                b.ox1 = std::min(s->nx, t.xe > 0 ? t.xe : t.x0 + 4 * (lanes - 2));
                b.oy0 = t.ya; b.oy1 = t.yb;
                if (t.flags & TASK_NOSTORE) b.ox1 = b.ox0;   // owns nothing
                bx.push_back(b);
            }
        }
        // boxes by (scene, first read column): a box can only meet boxes whose
        // columns start within one strip of its own
        std::map<std::pair<int, int>, std::vector<int>> by_col;
        for (size_t q = 0; q < bx.size(); q++) by_col[{bx[q].scene, bx[q].rx0}].push_back((int)q);
        auto meets = [](int a0, int a1, int b0, int b1) { return a0 < b1 && b0 < a1; };
        std::vector<std::vector<int>> deps(pitems.size());
        for (const Box& a : bx) {
            auto lo = by_col.lower_bound({a.scene, a.rx0 - STRIP});
            auto hi = by_col.upper_bound({a.scene, a.rx1});
            for (auto itr = lo; itr != hi; ++itr)
                for (int q : itr->second) {
                    const Box& b = bx[q];
                    if ((meets(a.rx0, a.rx1, b.ox0, b.ox1) && meets(a.ry0, a.ry1, b.oy0, b.oy1)) ||
                        (meets(a.ox0, a.ox1, b.rx0, b.rx1) && meets(a.oy0, a.oy1, b.ry0, b.ry1)))
                        deps[a.item].push_back(b.item);
                }
        }
        for (size_t i = 0; i < pitems.size(); i++) {
            std::vector<int>& d = deps[i];
            d.push_back((int)i);   // its own previous block
            std::sort(d.begin(), d.end());
            d.erase(std::unique(d.begin(), d.end()), d.end());
            dep_idx.insert(dep_idx.end(), d.begin(), d.end());
            dep_off[i + 1] = (int)dep_idx.size();
        }
    }
    dfree(c->d_scenes); dfree(c->d_tasks); dfree(c->d_tasks_b); dfree(c->d_samp); dfree(c->d_samp_scene); dfree(c->d_samp_off);
    dfree(c->d_ptasks); dfree(c->d_pitems); dfree(c->d_dep_off); dfree(c->d_dep_idx); dfree(c->d_done);
    dfree(c->d_pq);
    c->d_ptasks = nullptr; c->d_pitems = nullptr; c->d_dep_off = nullptr; c->d_dep_idx = nullptr; c->d_done = nullptr;
    c->d_pq = nullptr;
    c->n_pitems = 0;
    c->n_pint = c->n_pgen = 0;
    dfree(c->d_tasks_l);
    dfree(c->d_tasks_s);
    dfree(c->d_tasks_bd);
    dfree(c->d_tasks_n);
    dfree(c->d_dft);
    c->d_tasks_n = nullptr;
    c->d_tasks_l = nullptr;
    c->d_tasks_s = nullptr;
    c->d_tasks_bd = nullptr;
    c->d_dft = nullptr;
    c->n_dft = 0;
    c->d_scenes = nullptr; c->d_tasks = nullptr; c->d_tasks_b = nullptr; c->d_samp = nullptr; c->d_samp_scene = nullptr;
    c->d_samp_off = nullptr;
    adj_patch_descriptors(c, dev.data());   // the design history being recorded, if any
    c->h_scenes = dev;
    int rc;
    if ((rc = dalloc(c, &c->d_scenes, dev.size() * sizeof(TmzDev), "scene descriptors"))) return rc;
    if ((rc = dalloc(c, &c->d_tasks, tasks.size() * sizeof(Task), "tasks"))) return rc;
    if ((rc = dalloc(c, &c->d_tasks_b, tasks_b.size() * sizeof(Task), "tasks"))) return rc;
    if ((rc = dalloc(c, &c->d_ptasks, ptasks.size() * sizeof(Task), "persistent tasks"))) return rc;
    if ((rc = dalloc(c, &c->d_pitems, pitems.size() * sizeof(int2), "persistent items"))) return rc;
    if ((rc = dalloc(c, &c->d_dep_off, dep_off.size() * sizeof(int), "persistent dependencies"))) return rc;
    if ((rc = dalloc(c, &c->d_dep_idx, dep_idx.size() * sizeof(int), "persistent dependencies"))) return rc;
    if ((rc = dalloc(c, &c->d_done, pitems.size() * sizeof(unsigned), "persistent completion counts"))) return rc;
    // the two queues: interior items (interior warps), then the rest (general warps)
    std::vector<int> pq;
    for (size_t i = 0; i < pitems.size(); i++)
        if (pitems[i].x == PITEM_INTERIOR) pq.push_back((int)i);
    c->n_pint = (int)pq.size();
    for (size_t i = 0; i < pitems.size(); i++)
        if (pitems[i].x != PITEM_INTERIOR) pq.push_back((int)i);
    c->n_pgen = (int)pq.size() - c->n_pint;
    if ((rc = dalloc(c, &c->d_pq, std::max<size_t>(1, pq.size()) * sizeof(int), "persistent queues"))) return rc;
    if (!pq.empty())
        CK(cudaMemcpyAsync(c->d_pq, pq.data(), pq.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream), "upload");
    if ((rc = dalloc(c, &c->d_tasks_l, tasks_l.size() * sizeof(Task), "tasks"))) return rc;
    if ((rc = dalloc(c, &c->d_tasks_s, tasks_s.size() * sizeof(Task), "tasks"))) return rc;
    if ((rc = dalloc(c, &c->d_tasks_bd, tasks_bd.size() * sizeof(Task), "tasks"))) return rc;
    if ((rc = dalloc(c, &c->d_tasks_n, tasks_n.size() * sizeof(Task), "tasks"))) return rc;
    if ((rc = dalloc(c, &c->d_samp, tsamp.size() * sizeof(Sample2), "samples"))) return rc;
    if ((rc = dalloc(c, &c->d_samp_scene, ssamp.size() * sizeof(Sample2), "samples"))) return rc;
    if ((rc = dalloc(c, &c->d_samp_off, soff.size() * sizeof(int), "sample offsets"))) return rc;
    CK(cudaMemcpyAsync(c->d_scenes, dev.data(), dev.size() * sizeof(TmzDev), cudaMemcpyHostToDevice, c->stream), "upload");
    if (!tasks.empty())
        CK(cudaMemcpyAsync(c->d_tasks, tasks.data(), tasks.size() * sizeof(Task), cudaMemcpyHostToDevice, c->stream), "upload");
    if (!tasks_b.empty())
        CK(cudaMemcpyAsync(c->d_tasks_b, tasks_b.data(), tasks_b.size() * sizeof(Task), cudaMemcpyHostToDevice, c->stream), "upload");
    if (!ptasks.empty()) {
        CK(cudaMemcpyAsync(c->d_ptasks, ptasks.data(), ptasks.size() * sizeof(Task), cudaMemcpyHostToDevice, c->stream), "upload");
        CK(cudaMemcpyAsync(c->d_pitems, pitems.data(), pitems.size() * sizeof(int2), cudaMemcpyHostToDevice, c->stream), "upload");
        CK(cudaMemcpyAsync(c->d_dep_idx, dep_idx.data(), dep_idx.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream), "upload");
    }
    CK(cudaMemcpyAsync(c->d_dep_off, dep_off.data(), dep_off.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream), "upload");
    if (!tasks_l.empty())
        CK(cudaMemcpyAsync(c->d_tasks_l, tasks_l.data(), tasks_l.size() * sizeof(Task), cudaMemcpyHostToDevice, c->stream), "upload");
    if (!tasks_s.empty())
        CK(cudaMemcpyAsync(c->d_tasks_s, tasks_s.data(), tasks_s.size() * sizeof(Task), cudaMemcpyHostToDevice, c->stream), "upload");
    if (!tasks_bd.empty())
        CK(cudaMemcpyAsync(c->d_tasks_bd, tasks_bd.data(), tasks_bd.size() * sizeof(Task), cudaMemcpyHostToDevice, c->stream), "upload");
    if (!tasks_n.empty())
        CK(cudaMemcpyAsync(c->d_tasks_n, tasks_n.data(), tasks_n.size() * sizeof(Task), cudaMemcpyHostToDevice, c->stream), "upload");
    if (!tsamp.empty())
        CK(cudaMemcpyAsync(c->d_samp, tsamp.data(), tsamp.size() * sizeof(Sample2), cudaMemcpyHostToDevice, c->stream), "upload");
    if (!ssamp.empty())
        CK(cudaMemcpyAsync(c->d_samp_scene, ssamp.data(), ssamp.size() * sizeof(Sample2), cudaMemcpyHostToDevice, c->stream), "upload");
    CK(cudaMemcpyAsync(c->d_samp_off, soff.data(), soff.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream), "upload");
    // DFT accumulators of every cell monitor, for one launch per T-step block
    std::vector<DftItem> items;
    for (const DftMon& m : c->mons) {
        if (m.plane_k >= 0) continue;
        const Scene2* s = c->s2[m.scene];
        for (int q = 0; q < m.n_cells; q++)
            for (int f = 0; f < m.n_freq; f++) {
                DftItem it;
                it.rec = s->d_rec;
                it.acc = m.d_acc + (size_t)q * m.n_freq + f;
                double fr = m.freqs[f] * s->dt;
                fr -= floor(fr);
                const double v = ldexp(fr, 64);
                it.inc = v >= 18446744073709551615.0 ? 0ull : (unsigned long long)v;
                it.dt = (float)s->dt;
                it.n_rec = (int)s->samples.size();
                it.slot = m.slot0 + q;
                it.pad = 0;
                items.push_back(it);
            }
    }
    if (!items.empty()) {
        if ((rc = dalloc(c, &c->d_dft, items.size() * sizeof(DftItem), "dft items"))) return rc;
        CK(cudaMemcpyAsync(c->d_dft, items.data(), items.size() * sizeof(DftItem), cudaMemcpyHostToDevice, c->stream), "upload");
    }
    CK(cudaStreamSynchronize(c->stream), "upload task list");
    c->n_dft = (int)items.size();
    c->n_tasks = (int)tasks.size();
    c->n_tasks_b = (int)tasks_b.size();
    c->n_pitems = (int)pitems.size();
    c->n_tasks_l = (int)tasks_l.size();
    c->n_tasks_s = (int)tasks_s.size();
    c->n_tasks_bd = (int)tasks_bd.size();
    c->n_tasks_n = (int)tasks_n.size();
    c->task_narrow = want_narrow ? 1 : 0;
    c->task_pers = c->opt_kernel == 2 ? 1 : 0;
    c->warps_l = warps_l;
    c->warps_b = warps_b;
    c->task_warps_b = warps_b;
    c->coef_sq = 1;
    for (const Scene2* s : c->s2) c->coef_sq = c->coef_sq && s->dx == s->dy;
    // bulk row copies: each interior task's field rows start on 16 bytes and its
    // 144-byte material window (from the 16-byte boundary at or below its first
    // column) stays inside the row
    c->use_bulk = c->opt_bulk && c->d_bulk_err != nullptr;
    for (const Task& t : tasks) {
        if (t.scene < 0) continue;
        const int cs0 = t.x0 - HALO + PAD_X;
        if ((cs0 * 4) % 16 != 0 || (cs0 & ~15) + STRIP + 16 > c->s2[t.scene]->pitch) c->use_bulk = 0;
    }
    c->task_tb = T;
    c->task_seg = seg;
    c->dirty = false;
    return FDTD_OK;
}

int field_slot_2d(int comp) {
    if (comp == FDTD_EZ) return F_EZ;
    if (comp == FDTD_HX) return F_HX;
    if (comp == FDTD_HY) return F_HY;
    return -1;
}

}  // namespace

namespace gem {
cudaError_t ensure_dyn_smem(const void* kernel, size_t bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> done;
    std::lock_guard<std::mutex> lock(mu);
    size_t& have = done[std::make_pair(dev, kernel)];
    if (bytes <= have) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}

// record/waveform capacity and device descriptors for the next n_steps
int step_prepare(fdtd_ctx* c, int64_t n_steps) {
    if (c->s2.empty()) return fail(c, FDTD_ESTATE, "no scene");
    int rc = ensure_capacity(c, c->t + n_steps);
    if (rc) return rc;
    if (c->dirty || c->task_seg != c->opt_segment || c->task_narrow != (c->opt_kernel != 1 ? 1 : 0) ||
        c->task_pers != (c->opt_kernel == 2 ? 1 : 0) || c->task_warps_b != c->opt_warps_b) {
        rc = rebuild(c, c->opt_tblock, c->opt_segment, c->opt_warps);
        if (rc) return rc;
    }
    return FDTD_OK;
}

bool ctx_has_slab(const fdtd_ctx* c) {
    for (const Scene2* s : c->s2)
        if (s->ghost) return true;
    return false;
}

// the arrays a halo carries: Ez, Hx, Hy, and with a CPML the four psi arrays
// (the x-slab ones run along every row; the y-slab ones matter where a cut
// lies within the layer)
static int halo_slots(const Scene2* s) { return s->npml > 0 ? F_COUNT2 : 3; }

// copy `ghost` whole rows starting at local row r0 of every halo array between
// the context's current buffers and a packed [slot][ghost][nx] buffer
static int halo_copy(fdtd_ctx* c, Scene2* s, int r0, float* packed, const float* in, int on_device) {
    const int ns = halo_slots(s);
    const size_t plane = (size_t)s->ghost * s->nx;
    for (int f = 0; f < ns; f++) {
        float* dev = s->fbuf[f][c->parity] + (size_t)(r0 + PAD_Y) * s->pitch + PAD_X;
        cudaError_t e;
        if (packed)
            e = cudaMemcpy2DAsync(packed + f * plane, (size_t)s->nx * sizeof(float), dev, (size_t)s->pitch * sizeof(float),
                                  (size_t)s->nx * sizeof(float), s->ghost,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
        else
            e = cudaMemcpy2DAsync(dev, (size_t)s->pitch * sizeof(float), in + f * plane, (size_t)s->nx * sizeof(float),
                                  (size_t)s->nx * sizeof(float), s->ghost,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "halo copy");
    }
    if (!on_device) CK(cudaStreamSynchronize(c->stream), "halo copy");
    return FDTD_OK;
}

// the slab of a single-scene slab context, or NULL with the error set
static Scene2* slab_of(fdtd_ctx* c, int side) {
    Scene2* s = cur2(c);
    if (!s || !s->ghost) {
        fail(c, FDTD_EINVAL, "not a slab sub-domain (fdtd_create_slab)");
        return nullptr;
    }
    if (side != 0 && side != 1) {
        fail(c, FDTD_EINVAL, "side must be 0 (lower cut) or 1 (upper cut)");
        return nullptr;
    }
    if ((side == 0 ? s->ghost_lo : s->ghost_hi) == 0) {
        fail(c, FDTD_EINVAL, "the slab has no neighbour on side %d (it holds the grid's %s row)", side,
             side == 0 ? "first" : "last");
        return nullptr;
    }
    return s;
}

}  // namespace gem

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int fdtd_create(const fdtd_grid* grid, double dx, double dt, double courant, const uint8_t* mat_idx,
                const fdtd_material* table, int n_mat, void* cuda_stream, fdtd_ctx** out) {
    NvtxRange nvtx("fdtd_create");
    if (!out) return FDTD_EINVAL;
    *out = nullptr;
    if (!grid) return FDTD_EINVAL;
    if (grid->dims == 3) return fdtd_create3(grid, dx, dt, courant, mat_idx, table, n_mat, cuda_stream, out);
    fdtd_ctx* c = ctx_new(cuda_stream);
    Scene2* s = nullptr;
    int rc = scene2_init(c, grid, dx, dt, courant, mat_idx, table, n_mat, &s);
    if (rc) {
        // keep the context alive so the caller can read the message
        *out = c;
        return rc;
    }
    c->s2.push_back(s);
    *out = c;
    return FDTD_OK;
}

int fdtd_create_batch(int n_scenes, const fdtd_grid* grids, const double* dx, const double* dt,
                      const uint8_t* const* mat_idx, const fdtd_material* const* tables, const int* n_mat,
                      void* cuda_stream, fdtd_ctx** out) {
    NvtxRange nvtx("fdtd_create_batch");
    if (!out) return FDTD_EINVAL;
    *out = nullptr;
    fdtd_ctx* c = ctx_new(cuda_stream);
    *out = c;
    if (n_scenes < 1 || !grids || !dx || !dt || !mat_idx || !tables || !n_mat)
        return fail(c, FDTD_EINVAL, "batch needs n_scenes >= 1 and non-NULL arrays");
    for (int k = 0; k < n_scenes; k++) {
        Scene2* s = nullptr;
        int rc = scene2_init(c, &grids[k], dx[k], dt[k], 0.99, mat_idx[k], tables[k], n_mat[k], &s);
        if (rc) {
            c->err = "scene " + std::to_string(k) + ": " + c->err;
            return rc;
        }
        c->s2.push_back(s);
    }
    return FDTD_OK;
}

int fdtd_create_slab(const fdtd_grid* grid, int j0, int j1, int ghost, double dx, double dt, double courant,
                     const uint8_t* mat_idx, const fdtd_material* table, int n_mat, void* cuda_stream,
                     fdtd_ctx** out) {
    NvtxRange nvtx("fdtd_create_slab");
    if (!out) return FDTD_EINVAL;
    *out = nullptr;
    if (!grid) return FDTD_EINVAL;
    fdtd_ctx* c = ctx_new(cuda_stream);
    *out = c;
    if (grid->dims != 2) return fail(c, FDTD_EINVAL, "slab sub-domains are 2D");
    SlabSpec sp{j0, j1, ghost};
    Scene2* s = nullptr;
    int rc = scene2_init(c, grid, dx, dt, courant, mat_idx, table, n_mat, &s, &sp);
    if (rc) return rc;
    c->s2.push_back(s);
    return FDTD_OK;
}

int64_t fdtd_halo_count(const fdtd_ctx* c) {
    if (!c || c->dims != 2 || c->s2.empty()) return 0;
    const Scene2* s = c->s2[c->cur];
    return s->ghost ? (int64_t)halo_slots(s) * s->ghost * s->nx : 0;
}

int fdtd_halo_export(fdtd_ctx* c, int side, float* buf, int on_device) {
    NvtxRange nvtx("fdtd_halo_export");
    if (!c) return FDTD_EINVAL;
    Scene2* s = slab_of(c, side);
    if (!s) return FDTD_EINVAL;
    if (!buf) return fail(c, FDTD_EINVAL, "NULL halo buffer");
    // the owned rows next to the cut: the neighbour's ghost rows
    const int r0 = side == 0 ? s->ghost_lo : s->ny - s->ghost_hi - s->ghost;
    return halo_copy(c, s, r0, buf, nullptr, on_device);
}

int fdtd_halo_import(fdtd_ctx* c, int side, const float* buf, int on_device) {
    NvtxRange nvtx("fdtd_halo_import");
    if (!c) return FDTD_EINVAL;
    Scene2* s = slab_of(c, side);
    if (!s) return FDTD_EINVAL;
    if (!buf) return fail(c, FDTD_EINVAL, "NULL halo buffer");
    const int r0 = side == 0 ? 0 : s->ny - s->ghost_hi;
    return halo_copy(c, s, r0, nullptr, buf, on_device);
}

int fdtd_slab_rows(const fdtd_ctx* c, int* j0, int* j1, int* row_offset) {
    if (!c || c->dims != 2 || c->s2.empty()) return FDTD_EINVAL;
    const Scene2* s = c->s2[c->cur];
    if (j0) *j0 = s->yoff + s->ghost_lo;
    if (j1) *j1 = s->yoff + s->ny - s->ghost_hi;
    if (row_offset) *row_offset = s->yoff;
    return FDTD_OK;
}

int fdtd_select_scene(fdtd_ctx* c, int scene) {
    if (!c) return FDTD_EINVAL;
    const int n = c->dims == 2 ? (int)c->s2.size() : (c->s3 ? 1 : 0);
    if (scene < 0 || scene >= n) return fail(c, FDTD_EINVAL, "scene %d outside 0..%d", scene, n - 1);
    c->cur = scene;
    return FDTD_OK;
}

int fdtd_num_scenes(const fdtd_ctx* c) {
    if (!c) return 0;
    return c->dims == 2 ? (int)c->s2.size() : (c->s3 ? 1 : 0);
}

void fdtd_destroy(fdtd_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (Scene2* s : c->s2) scene2_free(s);
    for (DftMon& m : c->mons) {
        dfree(m.d_freq);
        dfree(m.d_acc);
        dfree(m.d_e1);
    }
    fdtd_destroy3(c);
    graph_free(c);
    adj_free(c);
    dfree(c->d_scenes); dfree(c->d_tasks); dfree(c->d_tasks_b); dfree(c->d_samp); dfree(c->d_samp_scene);
    dfree(c->d_samp_off);
    dfree(c->d_ptasks); dfree(c->d_pitems); dfree(c->d_dep_off); dfree(c->d_dep_idx); dfree(c->d_done);
    dfree(c->d_pq);
    dfree(c->d_dft);
    dfree(c->d_ctl);
    if (c->h_err) cudaFreeHost(c->h_err);
    dfree(c->d_bad);
    dfree(c->d_bulk_err);
    if (c->h_bad) cudaFreeHost(c->h_bad);
    if (c->graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)c->graph_exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    dfree(c->d_tasks_l);
    dfree(c->d_tasks_s);
    dfree(c->d_tasks_bd);
    dfree(c->d_tasks_n);
    if (c->aux) cudaStreamDestroy(c->aux);
    if (c->aux2) cudaStreamDestroy(c->aux2);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_join2) cudaEventDestroy(c->ev_join2);
    delete c;
}

const char* fdtd_last_error(const fdtd_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

int fdtd_set_option(fdtd_ctx* c, int option, int64_t v) {
    if (!c) return FDTD_EINVAL;
    switch (option) {
        case FDTD_OPT_KERNEL:
            if (v < 0 || v > 2) return fail(c, FDTD_EINVAL, "kernel option %lld outside 0..2", (long long)v);
            c->opt_kernel = (int)v;
            return FDTD_OK;
        case FDTD_OPT_GRAPH:
            if (v < 0 || v > 1) return fail(c, FDTD_EINVAL, "graph option must be 0 or 1");
            c->opt_graph = (int)v;
            return FDTD_OK;
        case FDTD_OPT_SPIN_LIMIT:
            if (v < 1) return fail(c, FDTD_EINVAL, "spin limit must be >= 1");
            c->spin_limit = v;
            return FDTD_OK;
        case FDTD_OPT_DEBUG_STALL_ITEM:
            if (v < -1 || v > (1 << 20)) return fail(c, FDTD_EINVAL, "debug item index out of range");
            c->opt_debug_skip = (int)v;
            return FDTD_OK;
        case FDTD_OPT_ADJ_STORE:
            if (v < 0 || v > 2) return fail(c, FDTD_EINVAL, "adjoint store option must be 0, 1 or 2");
            c->opt_adj_store = (int)v;
            return FDTD_OK;
        case FDTD_OPT_TBLOCK:
            if (v < 1 || v > (c->dims == 3 ? 2 : MAX_TB))
                return fail(c, FDTD_EINVAL, "tblock %lld outside 1..%d", (long long)v, c->dims == 3 ? 2 : MAX_TB);
            c->opt_tblock = (int)v;
            return FDTD_OK;
        case FDTD_OPT_SEGMENT:
            // 2D: rows per warp task (>= 8); 3D: planes per z-segment (>= 1; 0 = automatic)
            if (c->dims == 3 ? (v < 0 || v > (1 << 20)) : (v < 8 || v > (1 << 20)))
                return fail(c, FDTD_EINVAL, "segment %lld: 2D needs >= 8, 3D >= 1 (or 0, automatic)", (long long)v);
            c->opt_segment = (int)v;
            c->dirty = true;
            return FDTD_OK;
        case FDTD_OPT_CHECK_EVERY:
            if (c->dims != 2) return fail(c, FDTD_EINVAL, "the periodic finite check covers 2D contexts");
            if (v < 0 || v > (1 << 30)) return fail(c, FDTD_EINVAL, "check interval %lld outside 0..2^30", (long long)v);
            if (v > 0 && !c->d_bad) {
                if (!c->h_bad) return fail(c, FDTD_ENOMEM, "no pinned host word for the finite check");
                int rc = dalloc(c, &c->d_bad, sizeof(int), "finite-check flag");
                if (rc) return rc;
                CK(cudaMemsetAsync(c->d_bad, 0, sizeof(int), c->stream), "finite-check flag");
            }
            c->opt_check_every = (int)v;
            if (c->graph_exec) {   // a recorded step sequence lacks (or has) the checks
                cudaGraphExecDestroy((cudaGraphExec_t)c->graph_exec);
                c->graph_exec = nullptr;
            }
            return FDTD_OK;
        case FDTD_OPT_SEGMENT_B:
            if (v != 0 && (v < 4 || v > (1 << 20)))
                return fail(c, FDTD_EINVAL, "boundary segment %lld: 0 (automatic) or >= 4 rows", (long long)v);
            c->opt_segment_b = (int)v;
            c->dirty = true;
            return FDTD_OK;
        case FDTD_OPT_TAPER:
            if (v < 0 || v > 60) return fail(c, FDTD_EINVAL, "taper %lld outside 0..60 percent", (long long)v);
            c->opt_taper = (int)v;
            c->dirty = true;
            return FDTD_OK;
        case FDTD_OPT_BULK:
            if (v < 0 || v > 1) return fail(c, FDTD_EINVAL, "bulk option must be 0 or 1");
            if (c->dims != 2) return fail(c, FDTD_EINVAL, "bulk row copies are a 2D option");
            if (v == 1 && !c->d_bulk_err) {
                int rc = dalloc(c, &c->d_bulk_err, sizeof(int), "bulk-copy error word");
                if (rc) return rc;
                CK(cudaMemsetAsync(c->d_bulk_err, 0, sizeof(int), c->stream), "bulk-copy error word");
            }
            c->opt_bulk = (int)v;
            c->dirty = true;
            return FDTD_OK;
        case FDTD_OPT_PLAYOUT:
            if (v < 0 || v > 4096) return fail(c, FDTD_EINVAL, "persistent layout %lld outside 0..4096", (long long)v);
            c->opt_playout = (int)v;
            if (c->graph_exec) {   // a recorded step sequence holds the other launch
                cudaGraphExecDestroy((cudaGraphExec_t)c->graph_exec);
                c->graph_exec = nullptr;
            }
            return FDTD_OK;
        case FDTD_OPT_WARPS_B:
            if (v < 1 || v > 8) return fail(c, FDTD_EINVAL, "CPML warps %lld outside 1..8", (long long)v);
            c->opt_warps_b = (int)v;
            c->dirty = true;
            return FDTD_OK;
        case FDTD_OPT_WARPS:
            if (v < 1 || v > 8) return fail(c, FDTD_EINVAL, "warps %lld outside 1..8", (long long)v);
            c->opt_warps = (int)v;
            c->dirty = true;
            return FDTD_OK;
    }
    return fail(c, FDTD_EINVAL, "unknown option %d", option);
}

int64_t fdtd_get_option(const fdtd_ctx* c, int option) {
    if (!c) return -1;
    switch (option) {
        case FDTD_OPT_KERNEL: return c->opt_kernel;
        case FDTD_OPT_TBLOCK: return c->opt_tblock;
        case FDTD_OPT_SEGMENT: return c->opt_segment;
        case FDTD_OPT_WARPS: return c->opt_warps;
        case FDTD_OPT_GRAPH: return c->opt_graph;
        case FDTD_OPT_SPIN_LIMIT: return c->spin_limit;
        case FDTD_OPT_DEBUG_STALL_ITEM: return c->opt_debug_skip;
        case FDTD_OPT_ADJ_STORE: return c->opt_adj_store;
        case FDTD_OPT_SEGMENT_B: return c->opt_segment_b;
        case FDTD_OPT_CHECK_EVERY: return c->opt_check_every;
        case FDTD_OPT_TAPER: return c->opt_taper;
        case FDTD_OPT_WARPS_B: return c->opt_warps_b;
        case FDTD_OPT_PLAYOUT: return c->opt_playout;
        case FDTD_OPT_BULK: return c->opt_bulk;
    }
    return -1;
}

int fdtd_set_source(fdtd_ctx* c, int kind, int i, int j, int k, int component, const double* params,
                    const float* samples, int64_t n_samples) {
    if (!c) return FDTD_EINVAL;
    if (c->dims == 3) return fdtd_set_source3(c, kind, i, j, k, component, params, samples, n_samples);
    if (component != FDTD_EZ) return fail(c, FDTD_EINVAL, "2D TMz sources drive Ez only");
    return fdtd_set_line_source(c, kind, i, j, j + 1, params, samples, n_samples);
}

int fdtd_set_line_source(fdtd_ctx* c, int kind, int i, int j0, int j1, const double* params, const float* samples,
                         int64_t n_samples) {
    if (!c) return FDTD_EINVAL;
    if (c->dims != 2) return fail(c, FDTD_EINVAL, "line sources are 2D only");
    Scene2* s = cur2(c);
    if (!s) return fail(c, FDTD_ESTATE, "no scene");
    const int jmin = s->yoff == 0 ? 1 : 0;   // row 0 of a slab above the grid's first row is not a wall
    if (i < 1 || i >= s->nx || j0 < jmin || j1 > s->ny || j1 <= j0)
        return fail(c, FDTD_EINVAL, "source cells (%d, %d..%d) outside 1..nx-1 x %d..ny-1", i, j0, j1 - 1, jmin);
    const int j = j0;
    if (kind < FDTD_SRC_RICKER || kind > FDTD_SRC_SINE) return fail(c, FDTD_EINVAL, "unknown source kind %d", kind);
    if (kind == FDTD_SRC_SAMPLED) {
        if (!samples || n_samples < 0) return fail(c, FDTD_EINVAL, "sampled source needs samples");
        s->src_samples.assign(samples, samples + n_samples);
    } else {
        if (!params || !(params[0] > 0)) return fail(c, FDTD_EINVAL, "source parameter must be > 0");
        s->src_param = params[0];
    }
    s->src_kind = kind;
    s->src_i = i;
    s->src_j = j;
    s->src_j1 = j1;
    s->src_cap = 0;   // regenerate the waveform table
    c->dirty = true;
    return FDTD_OK;
}

int fdtd_set_materials(fdtd_ctx* c, const uint8_t* mat, const fdtd_material* table, int n_mat) {
    if (!c) return FDTD_EINVAL;
    Scene2* s = cur2(c);
    if (!s) return fail(c, FDTD_EINVAL, "fdtd_set_materials covers 2D scenes");
    if (!mat || !table) return fail(c, FDTD_EINVAL, "NULL material map or table");
    if (n_mat < 1 || n_mat > 255) return fail(c, FDTD_EINVAL, "n_mat %d outside 1..255", n_mat);
    for (int m = 0; m < n_mat; m++) {
        if (!(table[m].eps_r > 0)) return fail(c, FDTD_EINVAL, "material %d: eps_r must be > 0", m);
        if (table[m].mu_r != 1.0) return fail(c, FDTD_EINVAL, "material %d: mu_r must be 1 (non-magnetic medium)", m);
        if (!(table[m].sigma >= 0)) return fail(c, FDTD_EINVAL, "material %d: sigma must be >= 0", m);
    }
    if (s->split) {
        // the split layer's coefficients are per-axis profiles of vacuum: scan the layer only
        for (int j = 0; j < s->ny; j++) {
            const bool yl = j < s->npml || j >= s->ny - s->npml;
            for (int i = 0; i < s->nx; i++) {
                if (!yl && i >= s->npml && i < s->nx - s->npml) {
                    i = s->nx - s->npml - 1;
                    continue;
                }
                const int m = mat[(size_t)j * s->nx + i];
                if (m >= n_mat || table[m].eps_r != 1.0 || table[m].sigma != 0.0)
                    return fail(c, FDTD_EINVAL, "split-field PML: cell (%d, %d) in the layer is not vacuum", i, j);
            }
        }
    }
    std::vector<float4> co(256, make_float4(0, 0, 0, 0));
    for (int m = 0; m < n_mat; m++) co[m] = e_coeffs(table[m].eps_r, table[m].sigma, s->dt, s->dx, s->dy);
    // the [ny][nx] map lands inside the padded layout; the walls are re-marked PEC
    CK(cudaMemcpy2DAsync(s->d_mat + (size_t)PAD_Y * s->pitch + PAD_X, s->pitch, mat, s->nx, s->nx, s->ny,
                         cudaMemcpyHostToDevice, c->stream), "upload material map");
    CK(cudaMemcpyAsync(s->d_coef, co.data(), 256 * sizeof(float4), cudaMemcpyHostToDevice, c->stream),
       "upload coefficients");
    int rc = pec_walls(c, s);
    if (rc) return rc;
    if (s->d_dsg) {
        rc = tmz_design_band(c, s);   // the band holds material coefficients outside the rectangle
        if (rc) return rc;
    }
    s->eps_r.assign(n_mat, 0.0);
    s->sigma.assign(n_mat, 0.0);
    for (int m = 0; m < n_mat; m++) {
        s->eps_r[m] = table[m].eps_r;
        s->sigma[m] = table[m].sigma;
    }
    graph_free(c);   // the edge-list weights hold the old coefficients
    return FDTD_OK;
}

int fdtd_set_design(fdtd_ctx* c, int i0, int j0, int w, int h, const double* eps_r, const double* sigma,
                    int on_device) {
    if (!c) return FDTD_EINVAL;
    Scene2* s = cur2(c);
    if (!s) return fail(c, FDTD_EINVAL, "design regions are 2D only");
    if (s->ghost) return fail(c, FDTD_EINVAL, "design regions cover whole grids, not slab sub-domains");
    if (!eps_r || w < 1 || h < 1 || i0 < 1 || j0 < 1 || i0 + w > s->nx || j0 + h > s->ny)
        return fail(c, FDTD_EINVAL, "design rectangle (%d, %d, %d, %d) must lie in 1..nx-1 x 1..ny-1", i0, j0, w, h);
    if (s->split && (split_layer_cell(i0, j0, s->nx, s->ny, s->npml) ||
                     split_layer_cell(i0 + w - 1, j0 + h - 1, s->nx, s->ny, s->npml)))
        return fail(c, FDTD_EINVAL, "the design rectangle must lie inside the split-field PML");
    if (c->adj && s->d_dsg && (s->dsg_w != w || s->dsg_h != h))
        return fail(c, FDTD_EINVAL, "the design rectangle's size is fixed while checkpointing is on "
                                    "(its history blocks are sized for it)");
    const size_t n = (size_t)w * h;
    std::vector<float4> co;
    std::vector<float> fac;
    if (!on_device) {
        co.resize(n);
        fac.resize(n);
        for (size_t q = 0; q < n; q++) {
            const double sg = sigma ? sigma[q] : 0.0;
            if (!(eps_r[q] > 0) || !(sg >= 0))
                return fail(c, FDTD_EINVAL, "design cell %zu: eps_r must be > 0, sigma >= 0", q);
            co[q] = e_coeffs(eps_r[q], sg, s->dt, s->dx, s->dy);
            fac[q] = (float)(-kEps0 / (kEps0 * eps_r[q] + sg * s->dt / 2.0));
        }
    }
    if (!s->d_dsg || s->dsg_w != w || s->dsg_h != h) {
        dfree(s->d_dsg);
        dfree(s->d_band);
        dfree(s->d_dsg_fac);
        s->d_dsg = nullptr;
        s->d_band = nullptr;
        s->d_dsg_fac = nullptr;
        int rc = dalloc(c, &s->d_dsg, n * sizeof(float4), "design coefficients");
        if (rc) return rc;
        rc = dalloc(c, &s->d_band, (size_t)3 * h * s->pitch * sizeof(float), "design band");
        if (rc) return rc;
        rc = dalloc(c, &s->d_dsg_fac, n * sizeof(float), "design gradient factor");
        if (rc) return rc;
        s->dsg_w = s->dsg_h = 0;   // sized, not yet valid
    }
    if (on_device) {
        // eq. (7) per cell on the device, straight from the caller's device arrays
        int bad = 0;
        int rc = tmz_design_coeffs(c, s, eps_r, sigma, n, &bad);
        if (rc) return rc;
        if (bad) {
            // the coefficients were partly overwritten: drop the rectangle
            dfree(s->d_dsg);
            dfree(s->d_band);
            dfree(s->d_dsg_fac);
            s->d_dsg = nullptr;
            s->d_band = nullptr;
            s->d_dsg_fac = nullptr;
            s->dsg_w = s->dsg_h = 0;
            c->dirty = true;
            graph_free(c);
            return fail(c, FDTD_EINVAL, "design: every eps_r must be > 0 and every sigma >= 0 "
                                        "(the design rectangle is removed)");
        }
    } else {
        CK(cudaMemcpyAsync(s->d_dsg, co.data(), n * sizeof(float4), cudaMemcpyHostToDevice, c->stream),
           "upload design");
        CK(cudaMemcpyAsync(s->d_dsg_fac, fac.data(), n * sizeof(float), cudaMemcpyHostToDevice, c->stream),
           "upload design");
    }
    s->dsg_i0 = i0; s->dsg_j0 = j0; s->dsg_w = w; s->dsg_h = h;
    int brc = tmz_design_band(c, s);
    if (brc) return brc;
    CK(cudaStreamSynchronize(c->stream), "upload design");
    c->dirty = true;
    graph_free(c);   // the edge-list weights hold the old coefficients
    return FDTD_OK;
}

int fdtd_add_probe(fdtd_ctx* c, int i, int j, int k, int component, int* probe_id) {
    if (!c || !probe_id) return FDTD_EINVAL;
    if (c->dims == 3) return fdtd_add_probe3(c, i, j, k, component, probe_id);
    Scene2* s = cur2(c);
    if (!s) return fail(c, FDTD_ESTATE, "no scene");
    if (c->t != 0) return fail(c, FDTD_ESTATE, "probes must be added before the first step (t = %lld)", (long long)c->t);
    const int f = field_slot_2d(component);
    if (f < 0) return fail(c, FDTD_EINVAL, "2D probes record Ez, Hx or Hy");
    if (i < 0 || i >= s->nx || j < 0 || j >= s->ny) return fail(c, FDTD_EINVAL, "probe cell (%d, %d) outside the grid", i, j);
    Sample2 sp;
    sp.i = i; sp.j = j; sp.comp = f; sp.slot = (int)s->samples.size();
    s->samples.push_back(sp);
    s->rec_cap = 0;
    dfree(s->d_rec);
    s->d_rec = nullptr;
    Probe p;
    p.scene = c->cur; p.slot = sp.slot; p.t_start = 0;
    c->probes.push_back(p);
    *probe_id = (int)c->probes.size() - 1;
    c->dirty = true;
    return FDTD_OK;
}

int fdtd_add_dft_monitor(fdtd_ctx* c, const int32_t* cells, int n_cells, const double* freqs, int n_freq, int* mon_id) {
    if (!c || !mon_id) return FDTD_EINVAL;
    if (c->dims == 3) return fdtd_add_dft_monitor3(c, cells, n_cells, freqs, n_freq, mon_id);
    Scene2* s = cur2(c);
    if (!s) return fail(c, FDTD_ESTATE, "no scene");
    if (c->t != 0) return fail(c, FDTD_ESTATE, "monitors must be added before the first step");
    if (!cells || n_cells < 1 || !freqs || n_freq < 1) return fail(c, FDTD_EINVAL, "monitor needs cells and frequencies");
    for (int q = 0; q < n_cells; q++) {
        const int i = cells[2 * q], j = cells[2 * q + 1];
        if (i < 0 || i >= s->nx || j < 0 || j >= s->ny) return fail(c, FDTD_EINVAL, "monitor cell (%d, %d) outside the grid", i, j);
    }
    for (int f = 0; f < n_freq; f++)
        if (!(freqs[f] >= 0)) return fail(c, FDTD_EINVAL, "frequencies must be >= 0");
    DftMon m;
    m.scene = c->cur; m.n_cells = n_cells; m.n_freq = n_freq; m.slot0 = (int)s->samples.size();
    m.freqs.assign(freqs, freqs + n_freq);
    m.t_start = 0; m.plane_k = -1; m.comp_mask = 0;
    m.d_freq = nullptr; m.d_acc = nullptr;
    int rc = dalloc(c, &m.d_freq, n_freq * sizeof(double), "dft freqs");
    if (rc) return rc;
    rc = dalloc(c, &m.d_acc, (size_t)n_cells * n_freq * sizeof(float4), "dft accumulators");
    if (rc) { dfree(m.d_freq); return rc; }
    CK(cudaMemcpyAsync(m.d_freq, freqs, n_freq * sizeof(double), cudaMemcpyHostToDevice, c->stream), "upload freqs");
    CK(cudaMemsetAsync(m.d_acc, 0, (size_t)n_cells * n_freq * sizeof(float4), c->stream), "dft memset");
    CK(cudaStreamSynchronize(c->stream), "dft monitor");
    for (int q = 0; q < n_cells; q++) {
        Sample2 sp;
        sp.i = cells[2 * q]; sp.j = cells[2 * q + 1]; sp.comp = F_EZ; sp.slot = (int)s->samples.size();
        s->samples.push_back(sp);
    }
    s->rec_cap = 0;
    dfree(s->d_rec);
    s->d_rec = nullptr;
    c->mons.push_back(m);
    *mon_id = (int)c->mons.size() - 1;
    c->dirty = true;
    return FDTD_OK;
}

int fdtd_add_dft_plane(fdtd_ctx* c, int k, int comp_mask, const double* freqs, int n_freq, int* mon_id) {
    if (!c || !mon_id) return FDTD_EINVAL;
    if (c->dims != 3) return fail(c, FDTD_EINVAL, "plane monitors are 3D only");
    return fdtd_add_dft_plane3(c, k, comp_mask, freqs, n_freq, mon_id);
}

static bool any_split(const fdtd_ctx* c) {
    for (const Scene2* s : c->s2)
        if (s->split) return true;
    return false;
}

// the launches of n_steps steps (no allocation: step_prepare ran before)
static int step_launches(fdtd_ctx* c, int64_t n_steps) {
    const int T = c->opt_tblock;
    int64_t left = n_steps;
    int rc = FDTD_OK;
    while (left > 0) {
        int done;
        rc = adj_checkpoint_if_due(c);
        if (rc) return rc;
        if (c->opt_kernel == 1 || (c->opt_kernel == 2 && any_split(c))) {
            // the persistent kernel has no split-field variant: unfused pair
            rc = tmz_naive_step(c, c->t);
            done = 1;
        } else if (c->opt_kernel == 2 && left >= T) {
            // as many whole T-blocks as fit before the next checkpoint, in one launch
            const int64_t span = std::min<int64_t>(left, adj_next_boundary(c, c->t));
            const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(span / T, c->ctl_words - 4));
            if (span < T) {
                done = (int)span;
                rc = tmz_fused_launch(c, done, c->opt_warps, c->t, c->parity);
                c->parity ^= 1;
            } else {
                done = nb * T;
                rc = tmz_persistent_launch(c, T, c->t, nb, c->parity);
                c->parity ^= (nb & 1);
            }
        } else {
            // a T-step block never crosses a checkpoint boundary
            done = (int)std::min<int64_t>(std::min<int64_t>(T, left), adj_next_boundary(c, c->t));
            rc = tmz_fused_launch(c, done, c->opt_warps, c->t, c->parity);
            c->parity ^= 1;
        }
        if (rc) return rc;
        if (adj_edge_mode(c) && (c->opt_kernel == 1 || any_split(c))) {
            // the unfused pair does not keep the design window itself
            rc = adj_edge_record(c, done);
            if (rc) return rc;
        }
        if (c->n_dft > 0) {
            rc = dft_items_launch(c, c->t, done);
            if (rc) return rc;
        }
        if (c->opt_check_every > 0 && (c->t + done) / c->opt_check_every > c->t / c->opt_check_every) {
            // a step count divisible by the interval ended inside this block: scan the
            // fields into the sticky flag, which fdtd_sync reports
            cudaError_t e = tmz_finite_launch(c, c->d_bad);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c->h_bad, c->d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "periodic finite check");
        }
        c->t += done;
        left -= done;
    }
    return FDTD_OK;
}

int fdtd_step(fdtd_ctx* c, int64_t n_steps) {
    NvtxRange nvtx("fdtd_step");
    if (!c) return FDTD_EINVAL;
    if (n_steps < 0) return fail(c, FDTD_EINVAL, "n_steps < 0");
    if (n_steps == 0) return FDTD_OK;
    if (c->dims == 3) return fdtd_step3(c, n_steps);
    for (const Scene2* s : c->s2)
        if (s->ghost && n_steps > s->ghost)
            return fail(c, FDTD_EINVAL, "a slab sub-domain advances at most %d steps (its ghost depth) between "
                                        "halo exchanges; asked for %lld", s->ghost, (long long)n_steps);
    int rc = step_prepare(c, n_steps);
    if (rc) return rc;
    if (c->opt_kernel == 2) {
        // control words: 4 + one work counter per T-block of the longest launch
        const int need = 4 + (int)std::min<int64_t>(n_steps / std::max(1, c->opt_tblock) + 1, 1 << 20);
        if (c->ctl_words < need) {
            // the error word (ctl[2]) is sticky until fdtd_sync reports it: carry a
            // timeout of an earlier launch over into the new words
            CK(cudaStreamSynchronize(c->stream), "sync before growing the control words");
            dfree(c->d_ctl);
            c->d_ctl = nullptr;
            c->ctl_words = 0;
            rc = dalloc(c, &c->d_ctl, (size_t)need * sizeof(unsigned), "persistent control words");
            if (rc) return rc;
            c->ctl_words = need;
            CK(cudaMemsetAsync(c->d_ctl, 0, (size_t)need * sizeof(unsigned), c->stream), "control words");
            if (c->h_err && *c->h_err)
                CK(cudaMemcpyAsync(c->d_ctl + 2, c->h_err, sizeof(int), cudaMemcpyHostToDevice, c->stream),
                   "control words");
        }
        if (!c->h_err) return fail(c, FDTD_ENOMEM, "no pinned host word for the persistent kernel");
    }
    if (!c->opt_graph) return step_launches(c, n_steps);
    if (c->adj) return fail(c, FDTD_EINVAL, "CUDA-graph stepping and checkpointing cannot be combined");
    // replay the recorded graph when it was made for this start step, length and parity
    if (c->graph_exec && c->graph_t == c->t && c->graph_n == n_steps && c->graph_parity == c->parity) {
        CK(cudaGraphLaunch((cudaGraphExec_t)c->graph_exec, c->stream), "graph launch");
        const int64_t t0 = c->t;
        c->t = t0 + n_steps;
        c->parity = c->graph_parity_after;
        c->launches += c->graph_launches;
        return FDTD_OK;
    }
    if (c->graph_exec) {
        cudaGraphExecDestroy((cudaGraphExec_t)c->graph_exec);
        c->graph_exec = nullptr;
    }
    // record: the legacy default stream cannot be captured, so use a private one
    cudaStream_t user = c->stream;
    if (!user) {
        if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "capture stream");
        CK(cudaStreamSynchronize(0), "capture stream");
        c->stream = c->cap_stream;
    }
    const int64_t t0 = c->t;
    const int p0 = c->parity;
    const int64_t l0 = c->launches;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        rc = step_launches(c, n_steps);
        e = cudaStreamEndCapture(c->stream, &g);
    }
    c->stream = user;
    if (e != cudaSuccess || rc) {
        if (g) cudaGraphDestroy(g);
        c->t = t0;
        c->parity = p0;
        return rc ? rc : fail(c, FDTD_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->t = t0;
        c->parity = p0;
        return fail(c, FDTD_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    c->graph_exec = ex;
    c->graph_t = t0;
    c->graph_n = n_steps;
    c->graph_parity = p0;
    c->graph_parity_after = c->parity;
    c->graph_launches = c->launches - l0;
    c->launches = l0;
    CK(cudaGraphLaunch(ex, c->stream), "graph launch");
    c->launches += c->graph_launches;
    return FDTD_OK;
}

int fdtd_sync(fdtd_ctx* c) {
    if (!c) return FDTD_EINVAL;
    CK(cudaStreamSynchronize(c->stream), "sync");
    if (c->h_err && *c->h_err) {
        // report once: clear the sticky device word and its host copy
        if (c->d_ctl) CK(cudaMemsetAsync(c->d_ctl + 2, 0, sizeof(unsigned), c->stream), "clear the error word");
        CK(cudaStreamSynchronize(c->stream), "sync");
        *c->h_err = 0;
        if (c->h_bad) *c->h_bad = 0;   // fields of a cut-short run: a timeout is the first thing to report
        if (c->d_bad) CK(cudaMemset(c->d_bad, 0, sizeof(int)), "clear the finite-check flag");
        return fail(c, FDTD_ETIMEOUT, "a wait of the persistent kernel for another work item gave up (spin limit %lld)",
                    (long long)c->spin_limit);
    }
    if (c->d_bulk_err) {
        int v = 0;
        CK(cudaMemcpy(&v, c->d_bulk_err, sizeof(int), cudaMemcpyDeviceToHost), "read the bulk-copy error word");
        if (v) {
            CK(cudaMemset(c->d_bulk_err, 0, sizeof(int)), "clear the bulk-copy error word");
            return fail(c, FDTD_ETIMEOUT, "a wait of the interior kernel for its bulk row copies gave up "
                                          "(spin limit %lld)", (long long)c->spin_limit);
        }
    }
    if (c->h_bad && *c->h_bad) {
        if (c->d_bad) CK(cudaMemset(c->d_bad, 0, sizeof(int)), "clear the finite-check flag");
        *c->h_bad = 0;
        return fail(c, FDTD_EUNSTABLE, "the periodic finite check found non-finite field values "
                                       "(FDTD_OPT_CHECK_EVERY %d)", c->opt_check_every);
    }
    return FDTD_OK;
}

// time candidate settings on the current scenes; keep the fastest
int fdtd_autotune(fdtd_ctx* c, int trial_steps, double* best_ms) {
    NvtxRange nvtx("fdtd_autotune");
    if (!c) return FDTD_EINVAL;
    if (c->dims != 2) return fail(c, FDTD_EINVAL, "autotuning covers the 2D kernels");
    if (trial_steps < 4) return fail(c, FDTD_EINVAL, "trial_steps must be >= 4");
    if (c->adj) return fail(c, FDTD_EINVAL, "disable checkpointing before autotuning");
    if (ctx_has_slab(c)) return fail(c, FDTD_EINVAL, "autotuning covers whole grids, not slab sub-domains");
    struct Cand { int kernel, T, seg, warps, warps_b, playout; };
    std::vector<Cand> cand;
    // the segment height sets how many CTAs a block launches, so the sweep is
    // fine-grained: a list that fills whole waves of the 152 SMs wins; the CPML
    // CTAs' width sets how many SMs they share with interior CTAs
    for (int T = 2; T <= MAX_TB; T++)
        for (int seg = 16; seg <= 96; seg += 4)
            for (int w : {2, 4, 8})
                for (int wb : {2, 4, 8}) cand.push_back({0, T, seg, w, wb, 0});
    if (!any_split(c))   // the persistent kernel has no split-field variant
        for (int T = 2; T <= MAX_TB; T++)
            for (int seg : {32, 64, 96, 128})
                for (int pl : {0, 24, 48, 64}) cand.push_back({2, T, seg, 8, 2, pl});
    const int graph = c->opt_graph;
    c->opt_graph = 0;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "autotune");
    CK(cudaEventCreate(&e1), "autotune");
    double best = 1e30;
    Cand win = {c->opt_kernel, c->opt_tblock, c->opt_segment, c->opt_warps, c->opt_warps_b, c->opt_playout};
    const int taper0 = c->opt_taper;
    c->opt_taper = 0;   // the coarse pass and the boundary pass run uniform segments
    int rc = FDTD_OK;
    auto time_of = [&](const Cand& k, int steps, double* per) {
        c->opt_kernel = k.kernel; c->opt_tblock = k.T; c->opt_segment = k.seg; c->opt_warps = k.warps;
        c->opt_warps_b = k.warps_b;
        c->opt_playout = k.playout;
        c->dirty = true;
        int r = fdtd_reset(c);
        if (!r) r = fdtd_step(c, k.T);   // warm-up (and build) outside the timing
        if (r) return r;
        cudaEventRecord(e0, c->stream);
        if ((r = fdtd_step(c, steps))) return r;
        cudaEventRecord(e1, c->stream);
        if ((r = fdtd_sync(c))) return r;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        *per = ms / steps;
        return FDTD_OK;
    };
    // coarse pass over every candidate, then the four fastest again, longer
    std::vector<std::pair<double, int>> coarse;
    for (size_t q = 0; q < cand.size() && rc == FDTD_OK; q++) {
        double per = 0;
        rc = time_of(cand[q], trial_steps, &per);
        coarse.push_back({per, (int)q});
    }
    std::sort(coarse.begin(), coarse.end());
    for (size_t q = 0; q < coarse.size() && q < 4 && rc == FDTD_OK; q++) {
        const Cand& k = cand[coarse[q].second];
        double per = 0, per2 = 0;
        rc = time_of(k, 4 * trial_steps, &per);
        if (rc == FDTD_OK) rc = time_of(k, 4 * trial_steps, &per2);
        per = std::min(per, per2);
        if (rc == FDTD_OK && per < best) {
            best = per;
            win = k;
        }
    }
    // then a joint local search over the segment height and the boundary
    // tasks' height (the automatic choice included) around the two best
    // (T, warps, CPML warps) settings of the coarse pass: a block ends at the
    // later of the CPML chains and the interior's last wave, the two heights
    // move both (how many CTAs each launch has, how long a CPML chain is), and
    // the landscape has cliffs a coarse pass with the automatic boundary
    // height does not see
    int win_b = c->opt_segment_b;
    if (rc == FDTD_OK && win.kernel == 0) {
        const int saved_b = c->opt_segment_b;
        c->opt_segment_b = 0;
        double base = 0, base2 = 0;
        rc = time_of(win, 4 * trial_steps, &base);
        if (rc == FDTD_OK) rc = time_of(win, 4 * trial_steps, &base2);
        base = std::min(base, base2);
        win_b = 0;
        std::vector<Cand> seeds;
        for (size_t q = 0; q < coarse.size() && seeds.size() < 2; q++) {
            const Cand& k = cand[coarse[q].second];
            if (k.kernel != 0) continue;
            bool seen = false;
            for (const Cand& o : seeds) seen = seen || (o.T == k.T && o.warps == k.warps && o.warps_b == k.warps_b);
            if (!seen) seeds.push_back(k);
        }
        struct Trial { double ms; Cand k; int b; };
        std::vector<Trial> trials;
        for (const Cand& sd : seeds)
            for (int ds : {-8, -4, 0, 4, 8})
                for (int b : {0, 4, 8, 12, 16, 20, 24, 28, 32}) {
                    if (rc != FDTD_OK) break;
                    Cand k = sd;
                    k.seg = sd.seg + ds;
                    if (k.seg < 8) continue;
                    c->opt_segment_b = b;
                    double per = 0;
                    rc = time_of(k, 4 * trial_steps, &per);
                    if (rc == FDTD_OK) trials.push_back({per, k, b});
                }
        std::sort(trials.begin(), trials.end(), [](const Trial& a, const Trial& b) { return a.ms < b.ms; });
        for (size_t q = 0; q < trials.size() && q < 3 && rc == FDTD_OK; q++) {
            c->opt_segment_b = trials[q].b;
            double per = 0, per2 = 0;
            rc = time_of(trials[q].k, 4 * trial_steps, &per);
            if (rc == FDTD_OK) rc = time_of(trials[q].k, 4 * trial_steps, &per2);
            per = std::min(per, per2);
            if (rc == FDTD_OK && per < 0.99 * base) {   // a clear gain over the incumbent
                base = per;
                win = trials[q].k;
                win_b = trials[q].b;
            }
        }
        if (rc != FDTD_OK) win_b = saved_b;
        best = std::min(best, base);
    }
    // then tapered interior lists (taller segments in front, half-height ones
    // behind them, run tallest first) for the winner's T and warps
    int win_taper = 0;
    if (rc == FDTD_OK && win.kernel == 0) {
        c->opt_segment_b = win_b;
        const Cand base_k = win;
        for (int tp : {10, 20, 30, 45}) {
            for (int ds : {0, 8, 16, 24}) {
                if (rc != FDTD_OK) break;
                Cand k = base_k;
                k.seg = base_k.seg + ds;
                c->opt_taper = tp;
                double per = 0, per2 = 0;
                rc = time_of(k, 4 * trial_steps, &per);
                if (rc == FDTD_OK) rc = time_of(k, 4 * trial_steps, &per2);
                per = std::min(per, per2);
                if (rc == FDTD_OK && per < 0.99 * best) {
                    best = per;
                    win_taper = tp;
                    win.seg = k.seg;
                }
            }
        }
        if (rc != FDTD_OK) win_taper = taper0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->opt_kernel = win.kernel; c->opt_tblock = win.T; c->opt_segment = win.seg; c->opt_warps = win.warps;
    c->opt_warps_b = win.warps_b;
    c->opt_playout = win.playout;
    c->opt_taper = win.kernel == 0 ? win_taper : taper0;
    c->opt_segment_b = win_b;
    c->opt_graph = graph;
    c->dirty = true;
    int rc2 = fdtd_reset(c);
    if (rc) return rc;
    if (best_ms) *best_ms = best;
    return rc2;
}

int fdtd_read_probe(fdtd_ctx* c, int probe_id, float* out, int64_t n) {
    if (!c || !out) return FDTD_EINVAL;
    if (c->dims == 3) return fdtd_read_probe3(c, probe_id, out, n);
    if (probe_id < 0 || probe_id >= (int)c->probes.size()) return fail(c, FDTD_EINVAL, "no probe %d", probe_id);
    if (n < 0 || n > c->t) return fail(c, FDTD_EINVAL, "asked for %lld samples, %lld recorded", (long long)n, (long long)c->t);
    if (n == 0) return FDTD_OK;
    const Probe& p = c->probes[probe_id];
    Scene2* s = c->s2[p.scene];
    const int nrec = (int)s->samples.size();
    CK(cudaMemcpy2DAsync(out, sizeof(float), s->d_rec + p.slot, (size_t)nrec * sizeof(float), sizeof(float), (size_t)n,
                         cudaMemcpyDeviceToHost, c->stream), "read probe");
    CK(cudaStreamSynchronize(c->stream), "read probe");
    return FDTD_OK;
}

int fdtd_read_dft(fdtd_ctx* c, int mon_id, float* re, float* im) {
    if (!c || !re || !im) return FDTD_EINVAL;
    if (mon_id < 0 || mon_id >= (int)c->mons.size()) return fail(c, FDTD_EINVAL, "no monitor %d", mon_id);
    const DftMon& m = c->mons[mon_id];
    if (m.plane_k >= 0) return fdtd_read_dft3(c, mon_id, re, im);
    const size_t n = (size_t)m.n_cells * m.n_freq;
    std::vector<float4> acc(n);
    CK(cudaMemcpyAsync(acc.data(), m.d_acc, n * sizeof(float4), cudaMemcpyDeviceToHost, c->stream), "read dft");
    CK(cudaStreamSynchronize(c->stream), "read dft");
    for (size_t q = 0; q < n; q++) {
        // Kahan: the running compensation holds the negated lost low part
        re[q] = (float)((double)acc[q].x - (double)acc[q].z);
        im[q] = (float)((double)acc[q].y - (double)acc[q].w);
    }
    return FDTD_OK;
}

int fdtd_get_field(fdtd_ctx* c, int component, float* out, int on_device) {
    if (!c || !out) return FDTD_EINVAL;
    if (c->dims == 3) return fdtd_get_field3(c, component, out, on_device);
    Scene2* s = cur2(c);
    if (!s) return fail(c, FDTD_ESTATE, "no scene");
    const int f = field_slot_2d(component);
    if (f < 0) return fail(c, FDTD_EINVAL, "2D fields are Ez, Hx, Hy");
    const float* src = s->fbuf[f][c->parity] + (size_t)PAD_Y * s->pitch + PAD_X;
    CK(cudaMemcpy2DAsync(out, (size_t)s->nx * sizeof(float), src, (size_t)s->pitch * sizeof(float),
                         (size_t)s->nx * sizeof(float), (size_t)s->ny,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream), "get field");
    CK(cudaStreamSynchronize(c->stream), "get field");
    return FDTD_OK;
}

int fdtd_set_field(fdtd_ctx* c, int component, const float* in, int on_device) {
    if (!c || !in) return FDTD_EINVAL;
    if (c->dims == 3) return fdtd_set_field3(c, component, in, on_device);
    Scene2* s = cur2(c);
    if (!s) return fail(c, FDTD_ESTATE, "no scene");
    const int f = field_slot_2d(component);
    if (f < 0) return fail(c, FDTD_EINVAL, "2D fields are Ez, Hx, Hy");
    float* dst = s->fbuf[f][c->parity] + (size_t)PAD_Y * s->pitch + PAD_X;
    CK(cudaMemcpy2DAsync(dst, (size_t)s->pitch * sizeof(float), in, (size_t)s->nx * sizeof(float),
                         (size_t)s->nx * sizeof(float), (size_t)s->ny,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream), "set field");
    CK(cudaStreamSynchronize(c->stream), "set field");
    return FDTD_OK;
}

int fdtd_reset(fdtd_ctx* c) {
    if (!c) return FDTD_EINVAL;
    if (c->dims == 3) return fdtd_reset3(c);
    for (Scene2* s : c->s2) {
        const size_t fb = (size_t)s->pitch * s->rows * sizeof(float);
        for (int f = 0; f < F_COUNT2; f++)
            for (int p = 0; p < 2; p++) CK(cudaMemsetAsync(s->fbuf[f][p], 0, fb, c->stream), "reset");
        if (s->d_rec) CK(cudaMemsetAsync(s->d_rec, 0, (size_t)s->rec_cap * s->samples.size() * sizeof(float), c->stream), "reset");
    }
    for (DftMon& m : c->mons)
        CK(cudaMemsetAsync(m.d_acc, 0, (size_t)m.n_cells * m.n_freq * sizeof(float4), c->stream), "reset");
    CK(cudaStreamSynchronize(c->stream), "reset");
    c->t = 0;
    c->parity = 0;
    return FDTD_OK;
}

int64_t fdtd_time_step(const fdtd_ctx* c) { return c ? c->t : -1; }
int64_t fdtd_launch_count(const fdtd_ctx* c) { return c ? c->launches : -1; }

int fdtd_save_state(fdtd_ctx* c, void* buf, size_t* bytes) {
    NvtxRange nvtx("fdtd_save_state");
    if (!c || !bytes) return FDTD_EINVAL;
    if (c->dims == 3) return fdtd_save_state3(c, buf, bytes);
    size_t need = 2 * sizeof(int64_t);
    for (Scene2* s : c->s2) {
        need += (size_t)F_COUNT2 * s->nx * s->ny * sizeof(float);
        need += (size_t)c->t * s->samples.size() * sizeof(float);
    }
    for (DftMon& m : c->mons) need += (size_t)m.n_cells * m.n_freq * sizeof(float4);
    if (!buf) {
        *bytes = need;
        return FDTD_OK;
    }
    if (*bytes < need) return fail(c, FDTD_EINVAL, "state buffer of %zu bytes, %zu needed", *bytes, need);
    char* p = (char*)buf;
    int64_t hdr[2] = {c->t, (int64_t)c->s2.size()};
    memcpy(p, hdr, sizeof(hdr));
    p += sizeof(hdr);
    for (Scene2* s : c->s2) {
        for (int f = 0; f < F_COUNT2; f++) {
            const float* src = s->fbuf[f][c->parity] + (size_t)PAD_Y * s->pitch + PAD_X;
            CK(cudaMemcpy2DAsync(p, (size_t)s->nx * sizeof(float), src, (size_t)s->pitch * sizeof(float),
                                 (size_t)s->nx * sizeof(float), (size_t)s->ny, cudaMemcpyDeviceToHost, c->stream), "save");
            p += (size_t)s->nx * s->ny * sizeof(float);
        }
        const size_t rb = (size_t)c->t * s->samples.size() * sizeof(float);
        if (rb) CK(cudaMemcpyAsync(p, s->d_rec, rb, cudaMemcpyDeviceToHost, c->stream), "save");
        p += rb;
    }
    for (DftMon& m : c->mons) {
        const size_t ab = (size_t)m.n_cells * m.n_freq * sizeof(float4);
        CK(cudaMemcpyAsync(p, m.d_acc, ab, cudaMemcpyDeviceToHost, c->stream), "save");
        p += ab;
    }
    CK(cudaStreamSynchronize(c->stream), "save");
    *bytes = need;
    return FDTD_OK;
}

int fdtd_load_state(fdtd_ctx* c, const void* buf, size_t bytes) {
    NvtxRange nvtx("fdtd_load_state");
    if (!c || !buf) return FDTD_EINVAL;
    if (c->dims == 3) return fdtd_load_state3(c, buf, bytes);
    if (bytes < 2 * sizeof(int64_t)) return fail(c, FDTD_EINVAL, "state buffer too small");
    int64_t hdr[2];
    memcpy(hdr, buf, sizeof(hdr));
    if (hdr[1] != (int64_t)c->s2.size()) return fail(c, FDTD_EINVAL, "state has %lld scenes, context %zu", (long long)hdr[1], c->s2.size());
    size_t need = sizeof(hdr);
    for (Scene2* s : c->s2)
        need += (size_t)F_COUNT2 * s->nx * s->ny * sizeof(float) + (size_t)hdr[0] * s->samples.size() * sizeof(float);
    for (DftMon& m : c->mons) need += (size_t)m.n_cells * m.n_freq * sizeof(float4);
    if (bytes < need) return fail(c, FDTD_EINVAL, "state buffer of %zu bytes, %zu needed", bytes, need);
    int rc = ensure_capacity(c, std::max<int64_t>(hdr[0], 1));
    if (rc) return rc;
    const char* p = (const char*)buf + sizeof(hdr);
    c->parity = 0;
    for (Scene2* s : c->s2) {
        for (int f = 0; f < F_COUNT2; f++) {
            float* dst = s->fbuf[f][0] + (size_t)PAD_Y * s->pitch + PAD_X;
            CK(cudaMemcpy2DAsync(dst, (size_t)s->pitch * sizeof(float), p, (size_t)s->nx * sizeof(float),
                                 (size_t)s->nx * sizeof(float), (size_t)s->ny, cudaMemcpyHostToDevice, c->stream), "load");
            p += (size_t)s->nx * s->ny * sizeof(float);
        }
        const size_t rb = (size_t)hdr[0] * s->samples.size() * sizeof(float);
        if (rb) CK(cudaMemcpyAsync(s->d_rec, p, rb, cudaMemcpyHostToDevice, c->stream), "load");
        p += rb;
    }
    for (DftMon& m : c->mons) {
        const size_t ab = (size_t)m.n_cells * m.n_freq * sizeof(float4);
        CK(cudaMemcpyAsync(m.d_acc, p, ab, cudaMemcpyHostToDevice, c->stream), "load");
        p += ab;
    }
    CK(cudaStreamSynchronize(c->stream), "load");
    c->t = hdr[0];
    return FDTD_OK;
}

int fdtd_check_finite(fdtd_ctx* c) {
    if (!c) return FDTD_EINVAL;
    if (c->dims == 3) return fdtd_check_finite3(c);
    if (c->dirty) {
        int rc = rebuild(c, c->opt_tblock, c->opt_segment, c->opt_warps);
        if (rc) return rc;
    }
    int bad = 0;
    int rc = tmz_finite_check(c, &bad);
    if (rc) return rc;
    return bad ? fail(c, FDTD_EUNSTABLE, "non-finite field values") : FDTD_OK;
}

}  // extern "C"

/*
 * FP64 CPU oracle for the FDTD leapfrog step of arXiv 2405.00814 ("GEM").
 *
 * TEST INFRASTRUCTURE.  Plain, slow, obviously correct cell loops in double
 * precision.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load this library; it shares no code with the CUDA path.
 *
 * What each part follows:
 *   or_coeffs_e         Sec. III-B, eq. (7): Ca = A_-/A_+, Cb = dt/(A_+ eps).
 *   or2_layer_h         eqs. (8)(9) rotated to TMz (Hx, Hy from curl Ez);
 *                       Prop. 2, first message-passing step.
 *   or2_layer_e         eq. (7) rotated to TMz (Ez from curl H);
 *                       Prop. 2, second step; ordering per Sec. III-B.
 *   or_cpml_axis        CPML of Roden & Gedney (2000) (the paper's own absorber
 *                       is Berenger's split field, Sec. III-C; the CPML is the
 *                       published replacement used by these workloads).
 *   or2_graph_*         the literal graph of Prop. 1 and the two layers of
 *                       Prop. 2, with CPML auxiliaries appended as extra nodes.
 *   or2_adjoint_*       reverse mode of the same linear recurrence (the paper
 *                       only notes the message functions are differentiable,
 *                       Sec. IV-A); transposed layers in reverse order.
 *   or3_*               the 3D Yee extension the paper says follows directly
 *                       (Sec. III-B, Sec. IV-A).
 * Parallel loops (OpenMP over rows) do not change any per-cell arithmetic.
 */
#include "fdtd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
static const double C0 = 299792458.0;
static const double MU0 = 4.0e-7 * OR_PI;

double or_mu0(void) { return MU0; }
double or_eps0(void) { return 1.0 / (MU0 * C0 * C0); }
double or_c0(void) { return C0; }

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* thread count of later parallel loops (timing only; results do not depend on it) */
void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------------------------------
 * eq. (7): E^{n+1} = (A_-/A_+) E^n + dt/(A_+ eps) curl H^{n+1/2},
 * A_-/+ = 1 -/+ sigma dt/(2 eps).
 * ------------------------------------------------------------------------- */
void or_coeffs_e(int64_t n, const double* eps_r, const double* sigma, double dt, double* ca,
                 double* cb) {
    const double eps0 = or_eps0();
    for (int64_t k = 0; k < n; k++) {
        const double eps = eps0 * eps_r[k];
        const double am = 1.0 - sigma[k] * dt / (2.0 * eps);
        const double ap = 1.0 + sigma[k] * dt / (2.0 * eps);
        ca[k] = am / ap;
        cb[k] = dt / (ap * eps);
    }
}

static void cpml_point(double rho, int npml, double smax, double dt, double m, double amax,
                       double kmax, double* b, double* c, double* k) {
    if (rho <= 0.0) {
        *b = 0.0;
        *c = 0.0;
        *k = 1.0;
        return;
    }
    const double x = rho / (double)npml;
    const double sig = smax * pow(x, m);
    const double kap = 1.0 + (kmax - 1.0) * pow(x, m);
    const double alp = amax * (1.0 - x);
    const double bb = exp(-(sig / kap + alp) * dt / or_eps0());
    *b = bb;
    *c = sig * (bb - 1.0) / (sig * kap + kap * kap * alp);
    *k = kap;
}

void or_cpml_axis(int n, int npml, double delta, double dt, double m, double alpha_max,
                  double kappa_max, double* bE, double* cE, double* kE, double* bH, double* cH,
                  double* kH) {
    const double eta0 = sqrt(MU0 / or_eps0());
    const double smax = 0.8 * (m + 1.0) / (eta0 * delta);
    for (int i = 0; i < n; i++) {
        double rE = 0.0, rH = 0.0;
        if (npml > 0) {
            const double xe = (double)i, xh = (double)i + 0.5;
            const double lo = (double)npml, hi = (double)(n - npml);
            if (xe < lo) rE = lo - xe;
            if (xe > hi) rE = xe - hi;
            if (xh < lo) rH = lo - xh;
            if (xh > hi) rH = xh - hi;
        }
        cpml_point(rE, npml, smax, dt, m, alpha_max, kappa_max, &bE[i], &cE[i], &kE[i]);
        cpml_point(rH, npml, smax, dt, m, alpha_max, kappa_max, &bH[i], &cH[i], &kH[i]);
    }
}

void or_waveform(int kind, double param, double dt, int64_t nsteps, double* out) {
    for (int64_t n = 0; n < nsteps; n++) {
        const double t = (double)(n + 1) * dt;
        double s = 0.0;
        if (kind == 0) {
            const double tau = t - 1.5 / param;
            const double a = OR_PI * OR_PI * param * param * tau * tau;
            s = (1.0 - 2.0 * a) * exp(-a);
        } else if (kind == 1) {
            const double tg = 1.0 / param, t0 = 4.0 * tg;
            const double u = (t - t0) / tg;
            s = exp(-u * u) * sin(2.0 * OR_PI * param * (t - t0));
        } else if (kind == 2) {
            const double tg = 1.0 / param, t0 = 4.0 * tg;
            const double u = (t - t0) / tg;
            s = exp(-u * u);
        } else if (kind == 3) {
            s = sin(2.0 * OR_PI * param * t);
        }
        out[n] = s;
    }
}

/* ===========================================================================
 * 2D TMz
 * ========================================================================= */
#define IDX2(i, j) ((int64_t)(j) * nx + (i))

/* layer 1 (eqs. (8)(9) rotated): every H node, ghost Ez = 0 beyond i|j = N-1 */
void or2_layer_h(const or2_problem* p, or2_state* s) {
    const int nx = p->nx, ny = p->ny;
    const double dbx = p->dt / (MU0 * p->dx), dby = p->dt / (MU0 * p->dy);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++) {
        for (int i = 0; i < nx; i++) {
            const int64_t c = IDX2(i, j);
            const double ez = s->ez[c];
            const double ez_up = (j + 1 < ny) ? s->ez[c + nx] : 0.0;
            const double ez_rt = (i + 1 < nx) ? s->ez[c + 1] : 0.0;
            const double dey = ez_up - ez;
            const double dex = ez_rt - ez;
            s->phxy[c] = p->bhy[j] * s->phxy[c] + p->chy[j] * dey;
            s->hx[c] = s->hx[c] - dby * (dey / p->khy[j] + s->phxy[c]);
            s->phyx[c] = p->bhx[i] * s->phyx[c] + p->chx[i] * dex;
            s->hy[c] = s->hy[c] + dbx * (dex / p->khx[i] + s->phyx[c]);
        }
    }
}

/* layer 2 (eq. (7) rotated): Ez at i, j >= 1; Ez(0, .) and Ez(., 0) stay zero (PEC) */
void or2_layer_e(const or2_problem* p, or2_state* s) {
    const int nx = p->nx, ny = p->ny;
    const double dx = p->dx, dy = p->dy;
#pragma omp parallel for schedule(static)
    for (int j = 1; j < ny; j++) {
        for (int i = 1; i < nx; i++) {
            const int64_t c = IDX2(i, j);
            const double dhy = s->hy[c] - s->hy[c - 1];
            const double dhx = s->hx[c] - s->hx[c - nx];
            s->pezx[c] = p->bex[i] * s->pezx[c] + p->cex[i] * dhy;
            s->pezy[c] = p->bey[j] * s->pezy[c] + p->cey[j] * dhx;
            s->ez[c] = p->ca[c] * s->ez[c] +
                       p->cb[c] * ((dhy / p->kex[i] + s->pezx[c]) / dx -
                                   (dhx / p->key[j] + s->pezy[c]) / dy);
        }
    }
}

static void or2_record(const or2_problem* p, const or2_state* s, int64_t n, int64_t row,
                       or2_monitors* m) {
    if (!m) return;
    const int nx = p->nx;
    for (int q = 0; q < m->n_samp; q++) {
        const int64_t c = IDX2(m->si[q], m->sj[q]);
        const double* f = m->scomp[q] == 0 ? s->ez : (m->scomp[q] == 1 ? s->hx : s->hy);
        m->samp[row * m->n_samp + q] = f[c];
    }
    for (int q = 0; q < m->n_dft; q++) {
        const double e = s->ez[IDX2(m->di[q], m->dj[q])];
        for (int f = 0; f < m->n_freq; f++) {
            const double ph = 2.0 * OR_PI * m->freq[f] * (double)(n + 1) * p->dt;
            m->dre[q * m->n_freq + f] += e * cos(ph) * p->dt;
            m->dim[q * m->n_freq + f] -= e * sin(ph) * p->dt;
        }
    }
}

int or2_run(const or2_problem* p, or2_state* s, int64_t n0, int64_t nsteps, or2_monitors* m) {
    const int nx = p->nx;
    for (int64_t k = 0; k < nsteps; k++) {
        const int64_t n = n0 + k;
        or2_layer_h(p, s);
        or2_layer_e(p, s);
        if (p->src_i >= 0 && p->src && n < p->src_len) {
            const int nj = p->src_nj > 0 ? p->src_nj : 1;
            for (int q = 0; q < nj; q++) s->ez[IDX2(p->src_i, p->src_j + q)] += p->src[n];
        }
        or2_record(p, s, n, k, m);
    }
    return 0;
}

double or2_energy(const or2_problem* p, const double* eps_cell, const or2_state* s,
                  const double* hx_prev, const double* hy_prev) {
    const int64_t n = (int64_t)p->nx * p->ny;
    const double eps0 = or_eps0();
    double w = 0.0;
    for (int64_t c = 0; c < n; c++) {
        w += eps0 * eps_cell[c] * s->ez[c] * s->ez[c];
        w += MU0 * (s->hx[c] * hx_prev[c] + s->hy[c] * hy_prev[c]);
    }
    return w * p->dx * p->dy;
}

/* ---------------------------------------------------------------------------
 * literal graph (Prop. 1 numbering, Prop. 2 layers)
 * ------------------------------------------------------------------------- */
typedef struct {
    int64_t base;        /* 3 nx ny */
    int64_t off[4];      /* first node of psi_Hxy, psi_Hyx, psi_Ezx, psi_Ezy */
    int64_t count[4];
    int64_t* idx[4];     /* per cell: node index or -1 */
    int64_t* cell[4];    /* per psi node: its cell */
} or2_psi_map;

static int psi_exists(const or2_problem* p, int type, int i, int j) {
    switch (type) {
        case 0: return p->bhy[j] != 0.0 || p->chy[j] != 0.0;
        case 1: return p->bhx[i] != 0.0 || p->chx[i] != 0.0;
        case 2: return i >= 1 && j >= 1 && (p->bex[i] != 0.0 || p->cex[i] != 0.0);
        default: return i >= 1 && j >= 1 && (p->bey[j] != 0.0 || p->cey[j] != 0.0);
    }
}

static int psi_map_build(const or2_problem* p, or2_psi_map* m) {
    const int nx = p->nx, ny = p->ny;
    const int64_t ncell = (int64_t)nx * ny;
    m->base = 3 * ncell;
    int64_t next = m->base;
    for (int t = 0; t < 4; t++) {
        m->idx[t] = (int64_t*)malloc(sizeof(int64_t) * ncell);
        m->cell[t] = (int64_t*)malloc(sizeof(int64_t) * (ncell > 0 ? ncell : 1));
        if (!m->idx[t] || !m->cell[t]) return -1;
        m->off[t] = next;
        int64_t cnt = 0;
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                const int64_t c = IDX2(i, j);
                if (psi_exists(p, t, i, j)) {
                    m->idx[t][c] = next + cnt;
                    m->cell[t][cnt] = c;
                    cnt++;
                } else {
                    m->idx[t][c] = -1;
                }
            }
        m->count[t] = cnt;
        next += cnt;
    }
    return 0;
}

static void psi_map_free(or2_psi_map* m) {
    for (int t = 0; t < 4; t++) {
        free(m->idx[t]);
        free(m->cell[t]);
    }
}

int64_t or2_node_index(const or2_problem* p, int kind, int i, int j) {
    const int64_t nx = p->nx;
    if (kind == 0) return 2 * (int64_t)i + 1 + nx * (3 * (int64_t)j + 1); /* t: Ez */
    if (kind == 1) return (int64_t)i + 3 * (int64_t)j * nx;                /* u: Hx */
    return 2 * (int64_t)i + nx * (3 * (int64_t)j + 1);                     /* q: Hy */
}

int64_t or2_graph_nodes(const or2_problem* p) {
    or2_psi_map m;
    if (psi_map_build(p, &m)) {
        psi_map_free(&m);
        return -1;
    }
    int64_t n = m.base + m.count[0] + m.count[1] + m.count[2] + m.count[3];
    psi_map_free(&m);
    return n;
}

typedef struct {
    int64_t* rowptr;
    int32_t* col;
    double* w;
    int64_t nnz;
} csr_builder;

static void emit(csr_builder* b, int64_t col, double w) {
    if (b->col) {
        b->col[b->nnz] = (int32_t)col;
        b->w[b->nnz] = w;
    }
    b->nnz++;
}

/* decode a field node into (kind, i, j): kind 0 t (Ez), 1 u (Hx), 2 q (Hy) */
static void decode_field(int64_t v, int nx, int* kind, int* i, int* j) {
    const int64_t row = v / (3 * (int64_t)nx);
    const int64_t r = v % (3 * (int64_t)nx);
    *j = (int)row;
    if (r < nx) {
        *kind = 1;
        *i = (int)r;
    } else {
        const int64_t r2 = r - nx;
        *kind = (r2 % 2 == 0) ? 2 : 0;
        *i = (int)(r2 / 2);
    }
}

int64_t or2_graph_layer(const or2_problem* p, int layer, int64_t* rowptr, int32_t* col, double* w) {
    or2_psi_map m;
    if (psi_map_build(p, &m)) {
        psi_map_free(&m);
        return -1;
    }
    const int nx = p->nx, ny = p->ny;
    const double dbx = p->dt / (MU0 * p->dx), dby = p->dt / (MU0 * p->dy);
    const int64_t n_nodes = m.base + m.count[0] + m.count[1] + m.count[2] + m.count[3];
    csr_builder b = {rowptr, col, w, 0};
#define T_(i, j) or2_node_index(p, 0, (i), (j))
#define U_(i, j) or2_node_index(p, 1, (i), (j))
#define Q_(i, j) or2_node_index(p, 2, (i), (j))
    for (int64_t v = 0; v < n_nodes; v++) {
        if (rowptr) rowptr[v] = b.nnz;
        if (v < m.base) {
            int kind, i, j;
            decode_field(v, nx, &kind, &i, &j);
            const int64_t c = IDX2(i, j);
            if (layer == 1 && kind == 1) { /* Hx(i,j), eq. (8) rotated */
                const double a = dby * (1.0 / p->khy[j] + p->chy[j]);
                emit(&b, v, 1.0);
                if (j + 1 < ny) emit(&b, T_(i, j + 1), -a);
                emit(&b, T_(i, j), a);
                if (m.idx[0][c] >= 0) emit(&b, m.idx[0][c], -dby * p->bhy[j]);
            } else if (layer == 1 && kind == 2) { /* Hy(i,j), eq. (9) rotated */
                const double a = dbx * (1.0 / p->khx[i] + p->chx[i]);
                emit(&b, v, 1.0);
                if (i + 1 < nx) emit(&b, T_(i + 1, j), a);
                emit(&b, T_(i, j), -a);
                if (m.idx[1][c] >= 0) emit(&b, m.idx[1][c], dbx * p->bhx[i]);
            } else if (layer == 2 && kind == 0 && i >= 1 && j >= 1) { /* Ez(i,j), eq. (7) */
                const double cb = p->cb[c];
                const double ax = cb / p->dx * (1.0 / p->kex[i] + p->cex[i]);
                const double ay = cb / p->dy * (1.0 / p->key[j] + p->cey[j]);
                emit(&b, v, p->ca[c]);
                emit(&b, Q_(i, j), ax);
                emit(&b, Q_(i - 1, j), -ax);
                emit(&b, U_(i, j), -ay);
                emit(&b, U_(i, j - 1), ay);
                if (m.idx[2][c] >= 0) emit(&b, m.idx[2][c], cb / p->dx * p->bex[i]);
                if (m.idx[3][c] >= 0) emit(&b, m.idx[3][c], -cb / p->dy * p->bey[j]);
            } else {
                emit(&b, v, 1.0); /* not updated by this layer */
            }
        } else {
            int t = 0;
            while (t < 3 && v >= m.off[t] + m.count[t]) t++;
            const int64_t c = m.cell[t][v - m.off[t]];
            const int i = (int)(c % nx), j = (int)(c / nx);
            if (layer == 1 && t == 0) {
                emit(&b, v, p->bhy[j]);
                if (j + 1 < ny) emit(&b, T_(i, j + 1), p->chy[j]);
                emit(&b, T_(i, j), -p->chy[j]);
            } else if (layer == 1 && t == 1) {
                emit(&b, v, p->bhx[i]);
                if (i + 1 < nx) emit(&b, T_(i + 1, j), p->chx[i]);
                emit(&b, T_(i, j), -p->chx[i]);
            } else if (layer == 2 && t == 2) {
                emit(&b, v, p->bex[i]);
                emit(&b, Q_(i, j), p->cex[i]);
                emit(&b, Q_(i - 1, j), -p->cex[i]);
            } else if (layer == 2 && t == 3) {
                emit(&b, v, p->bey[j]);
                emit(&b, U_(i, j), p->cey[j]);
                emit(&b, U_(i, j - 1), -p->cey[j]);
            } else {
                emit(&b, v, 1.0);
            }
        }
    }
    if (rowptr) rowptr[n_nodes] = b.nnz;
#undef T_
#undef U_
#undef Q_
    psi_map_free(&m);
    return b.nnz;
}

void or2_state_to_nodes(const or2_problem* p, const or2_state* s, double* h) {
    or2_psi_map m;
    psi_map_build(p, &m);
    const int nx = p->nx, ny = p->ny;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            const int64_t c = IDX2(i, j);
            h[or2_node_index(p, 0, i, j)] = s->ez[c];
            h[or2_node_index(p, 1, i, j)] = s->hx[c];
            h[or2_node_index(p, 2, i, j)] = s->hy[c];
        }
    const double* psi[4] = {s->phxy, s->phyx, s->pezx, s->pezy};
    for (int t = 0; t < 4; t++)
        for (int64_t k = 0; k < m.count[t]; k++) h[m.off[t] + k] = psi[t][m.cell[t][k]];
    psi_map_free(&m);
}

void or2_nodes_to_state(const or2_problem* p, const double* h, or2_state* s) {
    or2_psi_map m;
    psi_map_build(p, &m);
    const int nx = p->nx, ny = p->ny;
    const int64_t ncell = (int64_t)nx * ny;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            const int64_t c = IDX2(i, j);
            s->ez[c] = h[or2_node_index(p, 0, i, j)];
            s->hx[c] = h[or2_node_index(p, 1, i, j)];
            s->hy[c] = h[or2_node_index(p, 2, i, j)];
        }
    double* psi[4] = {s->phxy, s->phyx, s->pezx, s->pezy};
    for (int t = 0; t < 4; t++) {
        memset(psi[t], 0, sizeof(double) * ncell);
        for (int64_t k = 0; k < m.count[t]; k++) psi[t][m.cell[t][k]] = h[m.off[t] + k];
    }
    psi_map_free(&m);
}

void or_csr_mv(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
               const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; r++) {
        double acc = 0.0;
        for (int64_t e = rowptr[r]; e < rowptr[r + 1]; e++) acc += w[e] * x[col[e]];
        y[r] = acc;
    }
}

void or_csr_mtv(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                const double* x, double* y) {
    for (int64_t r = 0; r < n; r++) y[r] = 0.0;
    for (int64_t r = 0; r < n; r++)
        for (int64_t e = rowptr[r]; e < rowptr[r + 1]; e++) y[col[e]] += w[e] * x[r];
}

/* ---------------------------------------------------------------------------
 * reverse mode.  Adjoint state a = (e, hx, hy, psi...) holds dL/d(state) after
 * a step; one call maps it to dL/d(state) before the step.
 * Layer 2 transposed, then layer 1 transposed.
 * ------------------------------------------------------------------------- */
static double g_x(const or2_problem* p, const or2_state* a, int i, int j) {
    /* coefficient of (Hy(i,j) - Hy(i-1,j)) gathered from E-layer rows at (i,j) */
    const int nx = p->nx, ny = p->ny;
    if (i < 1 || j < 1 || i >= nx || j >= ny) return 0.0;
    const int64_t c = IDX2(i, j);
    return p->cb[c] / p->dx * (1.0 / p->kex[i] + p->cex[i]) * a->ez[c] + p->cex[i] * a->pezx[c];
}

static double g_y(const or2_problem* p, const or2_state* a, int i, int j) {
    /* coefficient of (Hx(i,j) - Hx(i,j-1)) */
    const int nx = p->nx, ny = p->ny;
    if (i < 1 || j < 1 || i >= nx || j >= ny) return 0.0;
    const int64_t c = IDX2(i, j);
    return -p->cb[c] / p->dy * (1.0 / p->key[j] + p->cey[j]) * a->ez[c] + p->cey[j] * a->pezy[c];
}

static double f_x(const or2_problem* p, const or2_state* a, int i, int j) {
    /* coefficient of (Ez(i+1,j) - Ez(i,j)) gathered from H-layer rows at (i,j) */
    const int nx = p->nx, ny = p->ny;
    if (i < 0 || j < 0 || i >= nx || j >= ny) return 0.0;
    const int64_t c = IDX2(i, j);
    const double dbx = p->dt / (MU0 * p->dx);
    return dbx * (1.0 / p->khx[i] + p->chx[i]) * a->hy[c] + p->chx[i] * a->phyx[c];
}

static double f_y(const or2_problem* p, const or2_state* a, int i, int j) {
    /* coefficient of (Ez(i,j+1) - Ez(i,j)) */
    const int nx = p->nx, ny = p->ny;
    if (i < 0 || j < 0 || i >= nx || j >= ny) return 0.0;
    const int64_t c = IDX2(i, j);
    const double dby = p->dt / (MU0 * p->dy);
    return -dby * (1.0 / p->khy[j] + p->chy[j]) * a->hx[c] + p->chy[j] * a->phxy[c];
}

void or2_adjoint_step(const or2_problem* p, or2_state* a) {
    const int nx = p->nx, ny = p->ny;
    const double dbx = p->dt / (MU0 * p->dx), dby = p->dt / (MU0 * p->dy);
    /* layer 2 transposed: H adjoints gather from E rows (old e, psi_E) ... */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            const int64_t c = IDX2(i, j);
            a->hy[c] += g_x(p, a, i, j) - g_x(p, a, i + 1, j);
            a->hx[c] += g_y(p, a, i, j) - g_y(p, a, i, j + 1);
        }
    /* ... then the E rows' own transposes (cellwise) */
#pragma omp parallel for schedule(static)
    for (int j = 1; j < ny; j++)
        for (int i = 1; i < nx; i++) {
            const int64_t c = IDX2(i, j);
            const double e = a->ez[c];
            a->pezx[c] = p->bex[i] * a->pezx[c] + p->bex[i] * (p->cb[c] / p->dx) * e;
            a->pezy[c] = p->bey[j] * a->pezy[c] - p->bey[j] * (p->cb[c] / p->dy) * e;
            a->ez[c] = p->ca[c] * e;
        }
    /* layer 1 transposed: E adjoints gather from H rows (old hx, hy, psi_H) ... */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            const int64_t c = IDX2(i, j);
            a->ez[c] += f_y(p, a, i, j - 1) - f_y(p, a, i, j) + f_x(p, a, i - 1, j) - f_x(p, a, i, j);
        }
    /* ... then the psi_H rows (H rows have self weight 1) */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            const int64_t c = IDX2(i, j);
            a->phxy[c] = p->bhy[j] * a->phxy[c] - dby * p->bhy[j] * a->hx[c];
            a->phyx[c] = p->bhx[i] * a->phyx[c] + dbx * p->bhx[i] * a->hy[c];
        }
}

static int state_alloc(or2_state* s, int64_t n) {
    double** f[7] = {&s->ez, &s->hx, &s->hy, &s->pezx, &s->pezy, &s->phxy, &s->phyx};
    for (int k = 0; k < 7; k++) {
        *f[k] = (double*)calloc((size_t)n, sizeof(double));
        if (!*f[k]) return -1;
    }
    return 0;
}

static void state_free(or2_state* s) {
    free(s->ez); free(s->hx); free(s->hy);
    free(s->pezx); free(s->pezy); free(s->phxy); free(s->phyx);
}

static void state_copy(or2_state* d, const or2_state* s, int64_t n) {
    memcpy(d->ez, s->ez, sizeof(double) * n);
    memcpy(d->hx, s->hx, sizeof(double) * n);
    memcpy(d->hy, s->hy, sizeof(double) * n);
    memcpy(d->pezx, s->pezx, sizeof(double) * n);
    memcpy(d->pezy, s->pezy, sizeof(double) * n);
    memcpy(d->phxy, s->phxy, sizeof(double) * n);
    memcpy(d->phyx, s->phyx, sizeof(double) * n);
}

int or2_adjoint_grad(const or2_problem* p, const double* eps_cell, const double* sig_cell,
                     int64_t nsteps, int64_t ckpt, int n_mon, const int* mi, const int* mj,
                     int n_freq, const double* freq, int di0, int dj0, int dw, int dh,
                     double* loss, double* fre, double* fim, double* grad) {
    const int nx = p->nx;
    const int64_t ncell = (int64_t)p->nx * p->ny;
    const int64_t nd = (int64_t)dw * dh;
    const double eps0 = or_eps0(), dt = p->dt;
    if (ckpt <= 0) return -1;
    const int64_t nseg = (nsteps + ckpt - 1) / ckpt;
    or2_state* cps = (or2_state*)calloc((size_t)nseg, sizeof(or2_state));
    or2_state s, a;
    if (!cps || state_alloc(&s, ncell) || state_alloc(&a, ncell)) return -2;
    for (int64_t k = 0; k < nseg; k++)
        if (state_alloc(&cps[k], ncell)) return -2;
    double* eseg = (double*)malloc(sizeof(double) * nd * ckpt);
    double* kseg = (double*)malloc(sizeof(double) * nd * ckpt);
    if (!eseg || !kseg) return -2;

    /* forward: checkpoints and the DFT F_m(f) */
    memset(fre, 0, sizeof(double) * n_mon * n_freq);
    memset(fim, 0, sizeof(double) * n_mon * n_freq);
    or2_monitors mon;
    memset(&mon, 0, sizeof(mon));
    mon.n_dft = n_mon; mon.di = mi; mon.dj = mj; mon.n_freq = n_freq; mon.freq = freq;
    mon.dre = fre; mon.dim = fim;
    for (int64_t sg = 0; sg < nseg; sg++) {
        state_copy(&cps[sg], &s, ncell);
        const int64_t a0 = sg * ckpt, len = (a0 + ckpt <= nsteps) ? ckpt : nsteps - a0;
        or2_run(p, &s, a0, len, &mon);
    }
    double L = 0.0;
    for (int q = 0; q < n_mon * n_freq; q++) L += fre[q] * fre[q] + fim[q] * fim[q];
    *loss = L;

    /* reverse */
    memset(grad, 0, sizeof(double) * nd);
    for (int64_t sg = nseg - 1; sg >= 0; sg--) {
        const int64_t a0 = sg * ckpt, len = (a0 + ckpt <= nsteps) ? ckpt : nsteps - a0;
        state_copy(&s, &cps[sg], ncell);
        for (int64_t k = 0; k < len; k++) {
            const int64_t n = a0 + k;
            or2_layer_h(p, &s);
            /* K^{n+1/2} and E^n over the design region, before layer 2 */
            for (int dj = 0; dj < dh; dj++)
                for (int dI = 0; dI < dw; dI++) {
                    const int i = di0 + dI, j = dj0 + dj;
                    const int64_t c = IDX2(i, j);
                    const double dhy = s.hy[c] - s.hy[c - 1];
                    const double dhx = s.hx[c] - s.hx[c - nx];
                    const double px = p->bex[i] * s.pezx[c] + p->cex[i] * dhy;
                    const double py = p->bey[j] * s.pezy[c] + p->cey[j] * dhx;
                    kseg[k * nd + (int64_t)dj * dw + dI] =
                        (dhy / p->kex[i] + px) / p->dx - (dhx / p->key[j] + py) / p->dy;
                    eseg[k * nd + (int64_t)dj * dw + dI] = s.ez[c];
                }
            or2_layer_e(p, &s);
            if (p->src_i >= 0 && p->src && n < p->src_len)
                for (int q = 0; q < (p->src_nj > 0 ? p->src_nj : 1); q++) s.ez[IDX2(p->src_i, p->src_j + q)] += p->src[n];
        }
        for (int64_t k = len - 1; k >= 0; k--) {
            const int64_t n = a0 + k; /* reversing step n: E^n -> E^{n+1} */
            /* dL/dE^{n+1} at the monitors */
            for (int q = 0; q < n_mon; q++) {
                double g = 0.0;
                for (int f = 0; f < n_freq; f++) {
                    const double ph = 2.0 * OR_PI * freq[f] * (double)(n + 1) * dt;
                    g += 2.0 * (fre[q * n_freq + f] * cos(ph) - fim[q * n_freq + f] * sin(ph)) * dt;
                }
                a.ez[IDX2(mi[q], mj[q])] += g;
            }
            /* dL/deps_r += lambda_E^{n+1} (dCa/deps_r E^n + dCb/deps_r K^{n+1/2}) */
            for (int dj = 0; dj < dh; dj++)
                for (int dI = 0; dI < dw; dI++) {
                    const int64_t c = IDX2(di0 + dI, dj0 + dj);
                    const double eps = eps0 * eps_cell[c];
                    const double den = eps + sig_cell[c] * dt / 2.0;
                    const double dcb = -eps0 * dt / (den * den);
                    const double dca = eps0 * sig_cell[c] * dt / (den * den);
                    const int64_t d = (int64_t)dj * dw + dI;
                    grad[d] += a.ez[c] * (dca * eseg[k * nd + d] + dcb * kseg[k * nd + d]);
                }
            or2_adjoint_step(p, &a);
        }
    }
    for (int64_t k = 0; k < nseg; k++) state_free(&cps[k]);
    free(cps);
    state_free(&s);
    state_free(&a);
    free(eseg);
    free(kseg);
    return 0;
}

/* ===========================================================================
 * 3D Yee
 * ========================================================================= */
#define IDX3(i, j, k) (((int64_t)(k) * ny + (j)) * nx + (i))

static void or3_layer_h(const or3_problem* p, or3_state* s) {
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const double cdt = p->dt / MU0;
    const int64_t sy = nx, sz = (int64_t)nx * ny;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                const int64_t c = IDX3(i, j, k);
                const double ex = s->ex[c], ey = s->ey[c], ez = s->ez[c];
                const double ex_j = (j + 1 < ny) ? s->ex[c + sy] : 0.0;
                const double ex_k = (k + 1 < nz) ? s->ex[c + sz] : 0.0;
                const double ey_i = (i + 1 < nx) ? s->ey[c + 1] : 0.0;
                const double ey_k = (k + 1 < nz) ? s->ey[c + sz] : 0.0;
                const double ez_i = (i + 1 < nx) ? s->ez[c + 1] : 0.0;
                const double ez_j = (j + 1 < ny) ? s->ez[c + sy] : 0.0;
                const double dezy = ez_j - ez, deyz = ey_k - ey;
                const double dexz = ex_k - ex, dezx = ez_i - ez;
                const double deyx = ey_i - ey, dexy = ex_j - ex;
                s->phxy[c] = p->bhy[j] * s->phxy[c] + p->chy[j] * dezy;
                s->phxz[c] = p->bhz[k] * s->phxz[c] + p->chz[k] * deyz;
                s->hx[c] -= cdt * ((dezy / p->khy[j] + s->phxy[c]) / p->dy -
                                   (deyz / p->khz[k] + s->phxz[c]) / p->dz);
                s->phyz[c] = p->bhz[k] * s->phyz[c] + p->chz[k] * dexz;
                s->phyx[c] = p->bhx[i] * s->phyx[c] + p->chx[i] * dezx;
                s->hy[c] -= cdt * ((dexz / p->khz[k] + s->phyz[c]) / p->dz -
                                   (dezx / p->khx[i] + s->phyx[c]) / p->dx);
                s->phzx[c] = p->bhx[i] * s->phzx[c] + p->chx[i] * deyx;
                s->phzy[c] = p->bhy[j] * s->phzy[c] + p->chy[j] * dexy;
                s->hz[c] -= cdt * ((deyx / p->khx[i] + s->phzx[c]) / p->dx -
                                   (dexy / p->khy[j] + s->phzy[c]) / p->dy);
            }
}

static void or3_layer_e(const or3_problem* p, or3_state* s) {
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const int64_t sy = nx, sz = (int64_t)nx * ny;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                const int64_t c = IDX3(i, j, k);
                const double ca = p->ca[c], cb = p->cb[c];
                if (j >= 1 && k >= 1) { /* Ex */
                    const double dhzy = s->hz[c] - s->hz[c - sy];
                    const double dhyz = s->hy[c] - s->hy[c - sz];
                    s->pexy[c] = p->bey[j] * s->pexy[c] + p->cey[j] * dhzy;
                    s->pexz[c] = p->bez[k] * s->pexz[c] + p->cez[k] * dhyz;
                    s->ex[c] = ca * s->ex[c] + cb * ((dhzy / p->key[j] + s->pexy[c]) / p->dy -
                                                     (dhyz / p->kez[k] + s->pexz[c]) / p->dz);
                }
                if (i >= 1 && k >= 1) { /* Ey */
                    const double dhxz = s->hx[c] - s->hx[c - sz];
                    const double dhzx = s->hz[c] - s->hz[c - 1];
                    s->peyz[c] = p->bez[k] * s->peyz[c] + p->cez[k] * dhxz;
                    s->peyx[c] = p->bex[i] * s->peyx[c] + p->cex[i] * dhzx;
                    s->ey[c] = ca * s->ey[c] + cb * ((dhxz / p->kez[k] + s->peyz[c]) / p->dz -
                                                     (dhzx / p->kex[i] + s->peyx[c]) / p->dx);
                }
                if (i >= 1 && j >= 1) { /* Ez */
                    const double dhyx = s->hy[c] - s->hy[c - 1];
                    const double dhxy = s->hx[c] - s->hx[c - sy];
                    s->pezx[c] = p->bex[i] * s->pezx[c] + p->cex[i] * dhyx;
                    s->pezy[c] = p->bey[j] * s->pezy[c] + p->cey[j] * dhxy;
                    s->ez[c] = ca * s->ez[c] + cb * ((dhyx / p->kex[i] + s->pezx[c]) / p->dx -
                                                     (dhxy / p->key[j] + s->pezy[c]) / p->dy);
                }
            }
}

int or3_run(const or3_problem* p, or3_state* s, int64_t n0, int64_t nsteps, or3_monitors* m) {
    const int nx = p->nx, ny = p->ny;
    double* ecomp[3] = {s->ex, s->ey, s->ez};
    double* allc[6] = {s->ex, s->ey, s->ez, s->hx, s->hy, s->hz};
    for (int64_t q = 0; q < nsteps; q++) {
        const int64_t n = n0 + q;
        or3_layer_h(p, s);
        or3_layer_e(p, s);
        if (p->src_i >= 0 && p->src && n < p->src_len)
            ecomp[p->src_comp][IDX3(p->src_i, p->src_j, p->src_k)] += p->src[n];
        if (!m) continue;
        for (int t = 0; t < m->n_samp; t++)
            m->samp[q * m->n_samp + t] = allc[m->scomp[t]][IDX3(m->si[t], m->sj[t], m->sk[t])];
        if (m->plane_k >= 0) {
            for (int f = 0; f < m->n_freq; f++) {
                const double ph = 2.0 * OR_PI * m->freq[f] * (double)(n + 1) * p->dt;
                const double cr = cos(ph) * p->dt, ci = sin(ph) * p->dt;
                for (int pc = 0; pc < m->n_pc; pc++) {
                    const double* e = ecomp[m->pcomp[pc]];
                    double* re = m->pre + ((int64_t)pc * m->n_freq + f) * nx * ny;
                    double* im = m->pim + ((int64_t)pc * m->n_freq + f) * nx * ny;
                    for (int64_t c = 0; c < (int64_t)nx * ny; c++) {
                        const double v = e[(int64_t)m->plane_k * nx * ny + c];
                        re[c] += v * cr;
                        im[c] -= v * ci;
                    }
                }
            }
        }
    }
    return 0;
}

double or3_energy(const or3_problem* p, const double* eps_cell, const or3_state* s,
                  const double* hx_prev, const double* hy_prev, const double* hz_prev) {
    const int64_t n = (int64_t)p->nx * p->ny * p->nz;
    const double eps0 = or_eps0();
    double w = 0.0;
    for (int64_t c = 0; c < n; c++) {
        w += eps0 * eps_cell[c] * (s->ex[c] * s->ex[c] + s->ey[c] * s->ey[c] + s->ez[c] * s->ez[c]);
        w += MU0 * (s->hx[c] * hx_prev[c] + s->hy[c] * hy_prev[c] + s->hz[c] * hz_prev[c]);
    }
    return w * p->dx * p->dy * p->dz;
}

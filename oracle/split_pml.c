/*
 * FP64 oracle, part 2: the paper's own absorbing boundary, Berenger's
 * split-field PML (Sec. III-C, eqs. (10)-(13)), in TMz and as the literal
 * 4-node-per-cell graph (Sec. IV-B).
 *
 * TEST INFRASTRUCTURE, like fdtd_oracle.c: only the tests, the smoke check and
 * the benchmark's CPU baseline load it.
 *
 * Rotated to TMz (Ey -> -Ez, Hx -> Hx, Hz -> Hy; x -> x, z -> y) the four split
 * equations read
 *   eps dEzx/dt + sigma_x  Ezx = dHy/dx,     eps dEzy/dt + sigma_y  Ezy = -dHx/dy,
 *   mu0 dHx/dt  + sigma*_y Hx  = -dEz/dy,    mu0 dHy/dt  + sigma*_x Hy  =  dEz/dx,
 * with Ez = Ezx + Ezy and the matched magnetic conductivity sigma* = sigma mu0/eps0.
 * (As printed, the magnetic loss terms carry the wrong axis on Hx and a
 * misprinted E term on Hz; Berenger's form, used here, damps each H component
 * with the conductivity of the axis its derivative runs along.)  Each equation is
 * discretised with the semi-implicit averaging of eq. (7):
 *   Ca = (1 - s dt/2e) / (1 + s dt/2e),  Cb = dt / (e (1 + s dt/2e)),
 * for the E parts with s = sigma_cell + sigma_axis, e = eps0 eps_r, and the same
 * with s = sigma*, e = mu0 for H.  The layer grades sigma(rho) = sigma_max
 * (rho/d)^m over d cells, sigma_max = 0.8 (m+1) / (eta0 delta), rho measured from
 * the inner interface, E nodes at integer and H nodes at half-integer depth, the
 * layer backed by the PEC walls.  A soft source adds to Ezx.
 */
#include <math.h>
#include <stdlib.h>

#include "fdtd_oracle.h"

#define SP_PI 3.14159265358979323846
#define IX(i, j) ((int64_t)(j) * nx + (i))

void or_split_axis(int n, int npml, double delta, double m, double* sE, double* sH) {
    const double mu0 = or_mu0(), eps0 = or_eps0();
    const double eta0 = sqrt(mu0 / eps0);
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
        sE[i] = npml > 0 ? smax * pow(rE / npml, m) : 0.0;
        sH[i] = npml > 0 ? smax * pow(rH / npml, m) : 0.0;
    }
}

/* eq. (7) for one node: conductivity s, permittivity (or permeability) e */
static void semi_implicit(double s, double e, double dt, double* a, double* b) {
    const double ap = 1.0 + s * dt / (2.0 * e);
    *a = (1.0 - s * dt / (2.0 * e)) / ap;
    *b = dt / (e * ap);
}

static void split_e_coeffs(const or2s_problem* p, int i, int j, double* cax, double* cbx, double* cay,
                           double* cby) {
    const int nx = p->nx;
    const int64_t c = IX(i, j);
    const double e = or_eps0() * p->eps_cell[c];
    semi_implicit(p->sig_cell[c] + p->sxe[i], e, p->dt, cax, cbx);
    semi_implicit(p->sig_cell[c] + p->sye[j], e, p->dt, cay, cby);
}

/* H damping: sigma* = sigma mu0 / eps0 with permeability mu0 */
static void split_h_coeffs(double s, double dt, double* da, double* db) {
    semi_implicit(s * or_mu0() / or_eps0(), or_mu0(), dt, da, db);
}

static double ez_of(const or2s_state* s, int64_t c) { return s->ezx[c] + s->ezy[c]; }

void or2s_layer_h(const or2s_problem* p, or2s_state* s) {
    const int nx = p->nx, ny = p->ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++) {
        double day, dby;
        split_h_coeffs(p->syh[j], p->dt, &day, &dby);
        for (int i = 0; i < nx; i++) {
            double dax, dbx;
            split_h_coeffs(p->sxh[i], p->dt, &dax, &dbx);
            const int64_t c = IX(i, j);
            const double ez = ez_of(s, c);
            const double ez_up = (j + 1 < ny) ? ez_of(s, c + nx) : 0.0;
            const double ez_rt = (i + 1 < nx) ? ez_of(s, c + 1) : 0.0;
            s->hx[c] = day * s->hx[c] - dby * (ez_up - ez) / p->dy;
            s->hy[c] = dax * s->hy[c] + dbx * (ez_rt - ez) / p->dx;
        }
    }
}

void or2s_layer_e(const or2s_problem* p, or2s_state* s) {
    const int nx = p->nx, ny = p->ny;
#pragma omp parallel for schedule(static)
    for (int j = 1; j < ny; j++) {
        for (int i = 1; i < nx; i++) {
            const int64_t c = IX(i, j);
            double cax, cbx, cay, cby;
            split_e_coeffs(p, i, j, &cax, &cbx, &cay, &cby);
            s->ezx[c] = cax * s->ezx[c] + cbx * (s->hy[c] - s->hy[c - 1]) / p->dx;
            s->ezy[c] = cay * s->ezy[c] - cby * (s->hx[c] - s->hx[c - nx]) / p->dy;
        }
    }
}

static void split_record(const or2s_problem* p, const or2s_state* s, int64_t n, int64_t row, or2_monitors* m) {
    if (!m) return;
    const int nx = p->nx;
    for (int q = 0; q < m->n_samp; q++) {
        const int64_t c = IX(m->si[q], m->sj[q]);
        const double v = m->scomp[q] == 0 ? ez_of(s, c) : (m->scomp[q] == 1 ? s->hx[c] : s->hy[c]);
        m->samp[row * m->n_samp + q] = v;
    }
    for (int q = 0; q < m->n_dft; q++) {
        const double e = ez_of(s, IX(m->di[q], m->dj[q]));
        for (int f = 0; f < m->n_freq; f++) {
            const double ph = 2.0 * SP_PI * m->freq[f] * (double)(n + 1) * p->dt;
            m->dre[q * m->n_freq + f] += e * cos(ph) * p->dt;
            m->dim[q * m->n_freq + f] -= e * sin(ph) * p->dt;
        }
    }
}

int or2s_run(const or2s_problem* p, or2s_state* s, int64_t n0, int64_t nsteps, or2_monitors* m) {
    const int nx = p->nx;
    for (int64_t k = 0; k < nsteps; k++) {
        const int64_t n = n0 + k;
        or2s_layer_h(p, s);
        or2s_layer_e(p, s);
        if (p->src_i >= 0 && p->src && n < p->src_len) {
            const int nj = p->src_nj > 0 ? p->src_nj : 1;
            for (int q = 0; q < nj; q++) s->ezx[IX(p->src_i, p->src_j + q)] += p->src[n];
        }
        split_record(p, s, n, k, m);
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * literal graph with absorbing boundaries (Sec. IV-B): 4 nx ny nodes,
 * u(i,j) = i + 4 j nx (Hx), q(i,j) = 3 i + nx (4 j + 1) (Hy),
 * tx(i,j) = 3 i + 1 + nx (4 j + 1) (Ezx), tz(i,j) = 3 i + 2 + nx (4 j + 1) (Ezy).
 * The Ezy neighbourhood takes u(i,j-1) (the printed u(i-1,k) is a typo: Ezy
 * follows the y derivative of Hx), and the H neighbourhoods take the forward
 * neighbours of eqs. (8)(9), as in the field-only graph.
 * ------------------------------------------------------------------------- */
int64_t or2s_node_index(int nx, int kind, int i, int j) {
    const int64_t n = nx;
    if (kind == 0) return (int64_t)i + 4 * (int64_t)j * n;          /* u: Hx */
    return 3 * (int64_t)i + (kind - 1) + n * (4 * (int64_t)j + 1);  /* q: Hy, tx: Ezx, tz: Ezy */
}

static void decode4(int64_t v, int nx, int* kind, int* i, int* j) {
    const int64_t row = v / (4 * (int64_t)nx), r = v % (4 * (int64_t)nx);
    *j = (int)row;
    if (r < nx) {
        *kind = 0;
        *i = (int)r;
    } else {
        *kind = 1 + (int)((r - nx) % 3);
        *i = (int)((r - nx) / 3);
    }
}

int64_t or2s_graph_layer(const or2s_problem* p, int layer, int64_t* rowptr, int32_t* col, double* w) {
    const int nx = p->nx, ny = p->ny;
    const int64_t n_nodes = 4 * (int64_t)nx * ny;
    int64_t nnz = 0;
#define EMIT(cc, ww)                         \
    do {                                     \
        if (col) {                           \
            col[nnz] = (int32_t)(cc);        \
            w[nnz] = (ww);                   \
        }                                    \
        nnz++;                               \
    } while (0)
    for (int64_t v = 0; v < n_nodes; v++) {
        if (rowptr) rowptr[v] = nnz;
        int kind, i, j;
        decode4(v, nx, &kind, &i, &j);
        if (layer == 1 && kind == 0) {            /* Hx(i,j) */
            double da, db;
            split_h_coeffs(p->syh[j], p->dt, &da, &db);
            const double a = db / p->dy;
            EMIT(v, da);
            if (j + 1 < ny) {
                EMIT(or2s_node_index(nx, 2, i, j + 1), -a);
                EMIT(or2s_node_index(nx, 3, i, j + 1), -a);
            }
            EMIT(or2s_node_index(nx, 2, i, j), a);
            EMIT(or2s_node_index(nx, 3, i, j), a);
        } else if (layer == 1 && kind == 1) {     /* Hy(i,j) */
            double da, db;
            split_h_coeffs(p->sxh[i], p->dt, &da, &db);
            const double a = db / p->dx;
            EMIT(v, da);
            if (i + 1 < nx) {
                EMIT(or2s_node_index(nx, 2, i + 1, j), a);
                EMIT(or2s_node_index(nx, 3, i + 1, j), a);
            }
            EMIT(or2s_node_index(nx, 2, i, j), -a);
            EMIT(or2s_node_index(nx, 3, i, j), -a);
        } else if (layer == 2 && (kind == 2 || kind == 3) && i >= 1 && j >= 1) {
            double cax, cbx, cay, cby;
            split_e_coeffs(p, i, j, &cax, &cbx, &cay, &cby);
            if (kind == 2) {                      /* Ezx(i,j) */
                EMIT(v, cax);
                EMIT(or2s_node_index(nx, 1, i, j), cbx / p->dx);
                EMIT(or2s_node_index(nx, 1, i - 1, j), -cbx / p->dx);
            } else {                              /* Ezy(i,j) */
                EMIT(v, cay);
                EMIT(or2s_node_index(nx, 0, i, j), -cby / p->dy);
                EMIT(or2s_node_index(nx, 0, i, j - 1), cby / p->dy);
            }
        } else {
            EMIT(v, 1.0);                         /* not updated by this layer */
        }
    }
    if (rowptr) rowptr[n_nodes] = nnz;
#undef EMIT
    return nnz;
}

void or2s_state_to_nodes(const or2s_problem* p, const or2s_state* s, double* h) {
    const int nx = p->nx, ny = p->ny;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            const int64_t c = IX(i, j);
            h[or2s_node_index(nx, 0, i, j)] = s->hx[c];
            h[or2s_node_index(nx, 1, i, j)] = s->hy[c];
            h[or2s_node_index(nx, 2, i, j)] = s->ezx[c];
            h[or2s_node_index(nx, 3, i, j)] = s->ezy[c];
        }
}

void or2s_nodes_to_state(const or2s_problem* p, const double* h, or2s_state* s) {
    const int nx = p->nx, ny = p->ny;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            const int64_t c = IX(i, j);
            s->hx[c] = h[or2s_node_index(nx, 0, i, j)];
            s->hy[c] = h[or2s_node_index(nx, 1, i, j)];
            s->ezx[c] = h[or2s_node_index(nx, 2, i, j)];
            s->ezy[c] = h[or2s_node_index(nx, 3, i, j)];
        }
}

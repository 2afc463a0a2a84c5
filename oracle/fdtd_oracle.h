/*
 * FP64 CPU oracle for the FDTD leapfrog step of "Solving Maxwell's Equations
 * with Non-Trainable Graph Neural Network Message Passing" (arXiv 2405.00814).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load this library.  It shares no code, header, table or helper
 * with the CUDA path; the two meet only at the seeded scene inputs.
 *
 * Conventions (2D TMz, obtained from the paper's TE equations (3)-(9) by the
 * right-handed rotation x'=x, y'=z, z'=-y, which maps Ey -> -Ez', Hx -> Hx',
 * Hz -> Hy'):
 *   arrays are [ny][nx], x fastest;  Ez(i,j) at (i dx, j dy),
 *   Hx(i,j) at (i, j+1/2),  Hy(i,j) at (i+1/2, j);
 *   PEC walls at i = 0, j = 0 (stored zeros, never updated) and at i = nx,
 *   j = ny (ghost zeros), so the cavity is exactly nx*dx by ny*dy.
 * 3D Yee: Ex at (i+1/2, j, k), Ey at (i, j+1/2, k), Ez at (i, j, k+1/2),
 *   Hx at (i, j+1/2, k+1/2), Hy at (i+1/2, j, k+1/2), Hz at (i+1/2, j+1/2, k);
 *   arrays [nz][ny][nx]; tangential E is zero on the walls i|j|k = 0 and N.
 */
#ifndef GEM_FDTD_ORACLE_H
#define GEM_FDTD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- constants and coefficient formulas ---------------------------------- */
double or_mu0(void);
double or_eps0(void);
double or_c0(void);

/* Eq. (7): A_-/+ = 1 -/+ sigma dt / (2 eps);  Ca = A_-/A_+,  Cb = dt/(A_+ eps),
 * eps = eps0 * eps_r.  n entries in, n entries out. */
void or_coeffs_e(int64_t n, const double* eps_r, const double* sigma, double dt,
                 double* ca, double* cb);

/* CPML (Roden & Gedney 2000) 1D profiles for one axis of n cells with an
 * npml-cell layer at each end, backed by the PEC wall.  E nodes sit at integer
 * positions i, H nodes at i + 1/2; depth is measured from the inner interface.
 * sigma = sigma_max (rho/d)^m with sigma_max = 0.8 (m+1) / (eta0 delta),
 * kappa = 1 + (kappa_max - 1)(rho/d)^m, alpha = alpha_max (1 - rho/d),
 * b = exp(-(sigma/kappa + alpha) dt / eps0), c = sigma (b - 1) / (sigma kappa + kappa^2 alpha).
 * Outside the layer b = c = 0 and kappa = 1. */
void or_cpml_axis(int n, int npml, double delta, double dt, double m, double alpha_max,
                  double kappa_max, double* bE, double* cE, double* kE,
                  double* bH, double* cH, double* kH);

/* Source waveforms s(t) at t = (n+1) dt, n = 0 .. nsteps-1.
 * kind 0 Ricker(f_peak): (1 - 2 pi^2 f^2 tau^2) exp(-pi^2 f^2 tau^2), tau = t - 1.5/f.
 * kind 1 Gaussian-modulated(f0): exp(-((t - t0)/tg)^2) sin(2 pi f0 (t - t0)), tg = 1/f0, t0 = 4 tg.
 * kind 2 Gaussian(f_max): exp(-((t - t0)/tg)^2), tg = 1/f_max, t0 = 4 tg.
 * kind 3 sinusoid(f): sin(2 pi f t). */
void or_waveform(int kind, double param, double dt, int64_t nsteps, double* out);

/* ---- 2D TMz ------------------------------------------------------------- */
typedef struct {
    int nx, ny;
    double dx, dy, dt;
    const double *ca, *cb;                                 /* [ny*nx] */
    const double *bex, *cex, *kex, *bhx, *chx, *khx;       /* [nx] */
    const double *bey, *cey, *key, *bhy, *chy, *khy;       /* [ny] */
    int src_i, src_j;                                      /* -1: no source */
    const double* src;                                     /* src[n] = s((n+1) dt) */
    int64_t src_len;
    int src_nj;                                            /* cells (src_i, src_j .. src_j + src_nj - 1); 0 = 1 */
} or2_problem;

typedef struct {
    double *ez, *hx, *hy;                                  /* [ny*nx] */
    double *pezx, *pezy, *phxy, *phyx;                     /* CPML psi, [ny*nx] */
} or2_state;

/* Samples of a field component (0 Ez, 1 Hx, 2 Hy) at cells, taken after every
 * step (after the source), and a running DFT of Ez at cells:
 * F(f) += Ez^{n} exp(-i 2 pi f n dt) dt, n = 1..N. */
typedef struct {
    int n_samp;
    const int *si, *sj, *scomp;
    double* samp;                 /* [nsteps][n_samp] */
    int n_dft;
    const int *di, *dj;
    int n_freq;
    const double* freq;
    double *dre, *dim;            /* [n_dft][n_freq], accumulated */
} or2_monitors;

/* Layer 1 (H from curl E, eqs. (8)(9)) then layer 2 (E from curl H, eq. (7)),
 * then the soft source; steps n0 .. n0+nsteps-1 (step n makes E^{n+1}). */
int or2_run(const or2_problem* p, or2_state* s, int64_t n0, int64_t nsteps, or2_monitors* m);
void or2_layer_h(const or2_problem* p, or2_state* s);
void or2_layer_e(const or2_problem* p, or2_state* s);

/* Discrete energy sum eps Ez^2 + mu0 (H^{n+1/2} . H^{n-1/2}) (times dx dy). */
double or2_energy(const or2_problem* p, const double* eps_cell, const or2_state* s,
                  const double* hx_prev, const double* hy_prev);

/* ---- 2D TMz with the paper's split-field PML (split_pml.c) -------------
 * Berenger's split field (Sec. III-C, eqs. (10)-(13), rotated to TMz): Ez =
 * Ezx + Ezy, each part damped by the conductivity of its derivative's axis,
 * H damped by the matched sigma* = sigma mu0 / eps0; semi-implicit averaging
 * of eq. (7) throughout.  Graded sigma(rho) = sigma_max (rho/d)^m,
 * sigma_max = 0.8 (m+1) / (eta0 delta); E nodes at integer, H nodes at
 * half-integer depth (sE, sH: [n]). */
void or_split_axis(int n, int npml, double delta, double m, double* sE, double* sH);

typedef struct {
    int nx, ny;
    double dx, dy, dt;
    const double *eps_cell, *sig_cell;                     /* [ny*nx] eps_r, sigma (S/m) */
    const double *sxe, *sxh;                               /* [nx] layer sigma at E nodes i, H nodes i+1/2 */
    const double *sye, *syh;                               /* [ny] */
    int src_i, src_j;                                      /* soft source added to Ezx; -1: none */
    const double* src;
    int64_t src_len;
    int src_nj;                                            /* line of src_nj cells along j; 0 = 1 */
} or2s_problem;

typedef struct {
    double *ezx, *ezy, *hx, *hy;                           /* [ny*nx]; Ez = ezx + ezy */
} or2s_state;

/* layer 1 then layer 2 then the source, steps n0 .. n0+nsteps-1; monitors see
 * Ez = Ezx + Ezy (component 0), Hx (1), Hy (2) */
int or2s_run(const or2s_problem* p, or2s_state* s, int64_t n0, int64_t nsteps, or2_monitors* m);
void or2s_layer_h(const or2s_problem* p, or2s_state* s);
void or2s_layer_e(const or2s_problem* p, or2s_state* s);

/* literal graph with absorbing boundaries (Sec. IV-B): 4 nodes per cell,
 * u(i,j) = i + 4 j nx (Hx), q(i,j) = 3 i + nx (4 j + 1) (Hy),
 * tx(i,j) = 3 i + 1 + nx (4 j + 1) (Ezx), tz(i,j) = 3 i + 2 + nx (4 j + 1) (Ezy);
 * kind 0 u, 1 q, 2 tx, 3 tz.  CSR by destination over all nodes (identity rows
 * for nodes a layer does not update); returns nnz. */
int64_t or2s_node_index(int nx, int kind, int i, int j);
int64_t or2s_graph_layer(const or2s_problem* p, int layer, int64_t* rowptr, int32_t* col, double* w);
void or2s_state_to_nodes(const or2s_problem* p, const or2s_state* s, double* h);
void or2s_nodes_to_state(const or2s_problem* p, const double* h, or2s_state* s);

/* ---- literal GEM graph (Prop. 1 and 2) ----------------------------------
 * Node numbering of Prop. 1 with k -> j:  u(i,j) = i + 3 j nx  (Hx),
 * q(i,j) = 2 i + nx (3 j + 1)  (Hy),  t(i,j) = 2 i + 1 + nx (3 j + 1)  (Ez),
 * followed by the CPML psi nodes (psi_Hxy, psi_Hyx, psi_Ezx, psi_Ezy, each in
 * row-major cell order over the cells whose profile is non-zero).
 * Layer l is stored as CSR by destination over ALL nodes: rows of nodes the
 * layer does not update are identity rows (Prop. 2: updated neurons stay
 * constant). */
int64_t or2_graph_nodes(const or2_problem* p);
/* Fills rowptr[n_nodes+1], col[nnz], w[nnz] when the pointers are non-NULL;
 * returns nnz (or -1 on error). */
int64_t or2_graph_layer(const or2_problem* p, int layer, int64_t* rowptr, int32_t* col, double* w);
void or2_state_to_nodes(const or2_problem* p, const or2_state* s, double* h);
void or2_nodes_to_state(const or2_problem* p, const double* h, or2_state* s);
int64_t or2_node_index(const or2_problem* p, int kind, int i, int j); /* kind 0 t, 1 u, 2 q */
void or_csr_mv(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
               const double* x, double* y);
void or_csr_mtv(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                const double* x, double* y);

/* ---- discrete adjoint (reverse mode of the 2D recurrence) -------------- */
/* One reverse step: the adjoint of layer 2, then the adjoint of layer 1, in
 * place on an adjoint state (same layout as or2_state). */
void or2_adjoint_step(const or2_problem* p, or2_state* a);

/* d L / d eps_r over a design rectangle for L = sum_m sum_f |F_m(f)|^2, where F
 * is the running DFT of Ez at monitor cells (conventions of or2_monitors).  The
 * problem's ca/cb must already hold the design's coefficients; eps_cell and
 * sig_cell are the per-cell eps_r and sigma (needed for dCa/deps, dCb/deps).
 * Forward from the zero state with checkpoints every ckpt steps, then segments
 * are recomputed newest first and reversed.  Returns 0 on success. */
int or2_adjoint_grad(const or2_problem* p, const double* eps_cell, const double* sig_cell,
                     int64_t nsteps, int64_t ckpt, int n_mon, const int* mi, const int* mj,
                     int n_freq, const double* freq, int di0, int dj0, int dw, int dh,
                     double* loss, double* fre, double* fim, double* grad);

/* ---- 3D Yee ------------------------------------------------------------- */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz, dt;
    const double *ca, *cb;                                 /* [nz*ny*nx] */
    const double *bex, *cex, *kex, *bhx, *chx, *khx;       /* [nx] */
    const double *bey, *cey, *key, *bhy, *chy, *khy;       /* [ny] */
    const double *bez, *cez, *kez, *bhz, *chz, *khz;       /* [nz] */
    int src_i, src_j, src_k, src_comp;                     /* comp 0..2 = Ex,Ey,Ez */
    const double* src;
    int64_t src_len;
} or3_problem;

typedef struct {
    double *ex, *ey, *ez, *hx, *hy, *hz;
    /* psi_<field><derivative axis> */
    double *pexy, *pexz, *peyz, *peyx, *pezx, *pezy;
    double *phxy, *phxz, *phyz, *phyx, *phzx, *phzy;
} or3_state;

/* samples: comp 0..5 = Ex,Ey,Ez,Hx,Hy,Hz at (i,j,k); DFT plane: the E
 * components listed in pcomp at k = plane_k, all (i,j), accumulated into
 * pre/pim [n_pc][n_freq][ny][nx]. */
typedef struct {
    int n_samp;
    const int *si, *sj, *sk, *scomp;
    double* samp;
    int plane_k, n_pc;
    const int* pcomp;
    int n_freq;
    const double* freq;
    double *pre, *pim;
} or3_monitors;

int or3_run(const or3_problem* p, or3_state* s, int64_t n0, int64_t nsteps, or3_monitors* m);
double or3_energy(const or3_problem* p, const double* eps_cell, const or3_state* s,
                  const double* hx_prev, const double* hy_prev, const double* hz_prev);

int or_num_threads(void);
void or_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif

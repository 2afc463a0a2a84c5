// Internal structures of the GB300 FDTD library (not part of the C ABI).
//
// Device layout of a 2D TMz scene.  Every field and CPML auxiliary is an FP32
// array of `rows` x `pitch` floats with PAD_Y zero rows below and above the grid
// and PAD_X zero columns to its left; cell (i, j) lives at
//     (j + PAD_Y) * pitch + (i + PAD_X).
// pitch is a multiple of 32 floats, so each row starts on a 128-byte line, and
// wide enough that the widest warp strip (128 columns from i = x0 - HALO) of the
// last strip stays inside the row.  Pad cells and the PEC wall cells (i = 0 or
// j = 0) carry material PEC_MAT, whose coefficients are Ca = Cb = 0: their Ez
// stays exactly zero, so the zero pads act as the ghost PEC nodes at i, j = N.
// Fields exist twice (ping-pong): a fused launch reads buffer `parity` and
// writes buffer 1 - parity, so halos read by one warp are never overwritten by
// another warp during the launch.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "gem_fdtd.h"

namespace gem {

// a named range on the host timeline for profilers (creation, stepping,
// reverse mode, checkpoints); costs a function call when no tool listens
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int PAD_X = 8;
constexpr int PAD_Y = 8;
constexpr int PEC_MAT = 255;
constexpr int MAX_TB = 4;       // deepest temporal blocking of the fused kernel
constexpr int STRIP = 128;      // columns loaded by one warp (4 per lane)
constexpr int HALO = 4;         // halo columns each side (one lane): T <= HALO

// field slots of a 2D scene
enum { F_EZ = 0, F_HX, F_HY, F_PEZX, F_PEZY, F_PHXY, F_PHYX, F_COUNT2 };

// sample (probe / DFT cell) of a 2D scene
struct Sample2 {
    int i, j, comp, slot;   // comp: 0 Ez, 1 Hx, 2 Hy; slot: column in the record buffer
};

// what a warp task of the fused kernel needs to know about its scene
struct TmzDev {
    float* f[F_COUNT2][2];      // fields and psi, ping-pong
    const uint8_t* mat;         // [rows][pitch]
    const float4* coef;         // [256] (Ca, Cb/dx, Cb/dy, 0)
    const float* prof;          // 4 x-profiles [pitch] (bEx cEx bHx cHx), then 4 y-profiles [rows]
    int nx, ny, pitch, rows;
    int has_pml;
    int split;                          // split-field PML depth (profiles hold Ca, Cb/d, Da, Db/d per axis)
    float dbx, dby;             // dt / (mu0 dx), dt / (mu0 dy)
    int src_i, src_j;           // soft source cell or -1 (a line: cells (src_i, src_j .. src_j1 - 1))
    int src_j1;
    const float* src_wave;      // src_wave[n] = s((n+1) dt)
    long long src_len;
    float* rec;                 // sample record [cap][n_rec]
    int n_rec;
    long long rec_cap;
    // continuous-permittivity design rectangle (overrides the table inside it)
    int dsg_i0, dsg_j0, dsg_w, dsg_h;   // dsg_w == 0: none
    const float4* dsg_coef;             // [dsg_h][dsg_w] (Ca, Cb/dx, Cb/dy, Cb)
    const float* dsg_band;              // [3][dsg_h][pitch]: Ca, Cb/dx, Cb/dy of every cell of the design rows
    // reverse mode: the forward pass (or a recompute) records r^n = E^{n+1} - E^n
    // over the design rectangle; the adjoint kernels inject dL/dE^{n+1} at the
    // monitor cells and keep dL/dE^{n+1} over the design rectangle, which a
    // reduction after each segment turns into dL/deps_r
    float* dsg_rec;                     // [steps][dsg_h * dsg_w], step n at n - dsg_rec_n0; in edge-weight
                                        // mode [steps][3][dsg_h + 2][dsg_w + 2]: Ez^{n+1}, Hx^{n+1/2},
                                        // Hy^{n+1/2} of the window one cell around the design
    long long dsg_rec_n0, dsg_rec_len;
    float* grad;                        // [dsg_h][dsg_w]
    float* adj_rec;                     // [steps][dsg_h * dsg_w]: dL/dE^{n+1}, step n at n - dsg_rec_n0
    int adj_edges;                      // 1: adj_rec is [steps][3][dsg_h * dsg_w]: dL/dE^{n+1},
                                        //    dL/dHx^{n+1/2}, dL/dHy^{n+1/2} (edge-weight gradients)
    const float* adj_src;               // [steps][n_adj]: dL/dE^{n+1} at adjoint source cells
    int n_adj;
    // rows a with a < pml_ylo or a >= pml_yhi may lie in a y-slab of the CPML
    // (npml and ny - npml for a whole grid; shifted by the row offset of a slab
    // sub-domain, whose CPML profile is the whole grid's)
    int pml_ylo, pml_yhi;
};

// one warp's work in the fused kernel: columns [x0, x0 + STRIP - 2 HALO) and
// rows [ya, yb) of one scene, plus the samples that fall in that output region
// (a narrow task of a lane group owns columns [x0, x0 + (NG_LANES - 2) 4))
struct Task {
    int scene;
    int x0, ya, yb;
    int samp_begin, samp_end;   // into the launch's Sample2 list
    int flags;                  // TASK_* bits
    int xe;                     // > 0: no column at or past xe is owned (0: none)
};
// TASK_NOSTORE: a copy that only fills a lane group of a warp (computes, stores nothing)
enum { TASK_PML = 1, TASK_SRC = 2, TASK_DSG = 4, TASK_NOSTORE = 8 };
// lanes per task of the narrow CPML kernel (4 tasks per warp); each owns
// NG_OWN columns at one side of the grid, the columns of an x-slab of the CPML
// and its reach (rebuild uses them when the layer is at most NG_OWN - HALO -
// MAX_TB cells deep, so that no interior strip computes a CPML cell it owns)
constexpr int NG_LANES = 8;
constexpr int NG_OWN = (NG_LANES - 2) * 4;
// kinds of persistent-kernel items
enum { PITEM_INTERIOR = 0, PITEM_GENERAL = 1, PITEM_NARROW = 2 };

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct DftMon {
    int scene;
    int n_cells, n_freq;
    int slot0;                  // record slots slot0 .. slot0 + n_cells - 1 (Ez at the cells)
    std::vector<double> freqs;
    double* d_freq;             // device copy
    float4* d_acc;              // [n_cells][n_freq] (re, im, comp_re, comp_im)
    int64_t t_start;            // first step accumulated
    // 3D plane monitor
    int plane_k, comp_mask;
    float* d_e1 = nullptr;      // 3D two-step kernel: the plane's E after the first step, [3][rows][pitch]
};

// one (cell, frequency) accumulator of a 2D cell monitor, for the single DFT
// launch per T-step block.  The phase of step n is (n + 1) * inc modulo 2^64,
// a 64-bit fixed-point fraction of a cycle (inc = frac(f dt) * 2^64).
struct DftItem {
    const float* rec;
    float4* acc;
    unsigned long long inc;
    float dt;
    int n_rec, slot, pad;
};

struct Probe {
    int scene, slot;
    int64_t t_start;
};

struct Scene2 {
    int nx, ny, pitch, rows, npml;
    int split;                           // 1: npml is a split-field PML, not a CPML
    double dx, dy, dt;
    std::vector<double> eps_r, sigma;    // material table
    float* fbuf[F_COUNT2][2];
    uint8_t* d_mat;
    float4* d_coef;
    float* d_prof;
    // source
    int src_kind, src_i, src_j, src_j1;
    double src_param;
    std::vector<float> src_samples;
    float* d_src;
    long long src_cap;
    // samples
    std::vector<Sample2> samples;
    float* d_rec;
    long long rec_cap;
    // design rectangle
    int dsg_i0, dsg_j0, dsg_w, dsg_h;
    float4* d_dsg;
    float* d_band;                       // see TmzDev::dsg_band
    float* d_dsg_fac;                    // [dsg_h][dsg_w]: -eps0 / (eps0 eps_r + sigma dt / 2), the
                                         // per-cell factor of the eps_r gradient (reverse mode)
    // y-slab sub-domain of a larger grid (fdtd_create_slab): local row r is row
    // r + yoff of the whole grid (ny_glob rows); ghost_lo / ghost_hi rows below /
    // above the owned rows are copies of the neighbours' rows, refreshed by
    // fdtd_halo_import; ghost is the depth of a halo (0: a whole grid)
    int yoff, ny_glob, ghost, ghost_lo, ghost_hi;
};

}  // namespace gem

struct Scene3;

struct fdtd_ctx {
    int dims;
    cudaStream_t stream;
    std::vector<gem::Scene2*> s2;
    Scene3* s3;
    int cur;
    int64_t t;
    int parity;
    std::vector<gem::Probe> probes;
    std::vector<gem::DftMon> mons;
    std::string err;
    int64_t launches;
    // options
    int opt_kernel, opt_tblock, opt_segment, opt_warps;
    int opt_segment_b;           // FDTD_OPT_SEGMENT_B (0: max(8, opt_segment / 2))
    int opt_taper;               // FDTD_OPT_TAPER: percent of interior rows in half-height tail segments
    int opt_warps_b;             // FDTD_OPT_WARPS_B: warps per CTA of the forward CPML kernels
    int opt_playout;             // FDTD_OPT_PLAYOUT: persistent CTAs (0: 12-warp; k: 16-warp, k general)
    // device copies for the fused kernel, rebuilt when dirty
    bool dirty;
    gem::TmzDev* d_scenes;
    gem::Task* d_tasks;
    gem::Task* d_tasks_b;          // CPML tasks (a slab within reach)
    int n_tasks_b, warps_b;
    gem::Task* d_tasks_s;          // tasks within reach of a split-field PML layer
    int n_tasks_s;
    gem::Task* d_tasks_bd;         // CPML tasks with a design rectangle in reach
    int n_tasks_bd;
    gem::Task* d_tasks_n;          // narrow x-slab CPML tasks, NG_LANES lanes each (4 per warp)
    int n_tasks_n;
    int task_narrow;               // the lists were built with narrow x-slab tasks (kernels 0, 2)
    int task_warps_b;              // the CPML lists are padded to CTAs of this many warps
    int coef_sq;                   // every scene has dx == dy: the interior kernel stages (Ca, Cb/dx)
    int opt_bulk;                  // FDTD_OPT_BULK: interior rows by cp.async.bulk
    int use_bulk;                  // opt_bulk and every interior task's rows suit the bulk copies
    int* d_bulk_err;               // sticky device word: a bulk-copy wait gave up
    int task_pers;                 // the persistent kernel's items were built (kernel 2)
    gem::Task* d_tasks_l;          // lite tasks: design, source, probes or ragged edge, no CPML
    int n_tasks_l, warps_l;
    cudaStream_t aux, aux2;        // forked streams for the CPML and lite tasks
    cudaEvent_t ev_fork, ev_join, ev_join2;
    gem::Sample2* d_samp;          // samples in task order (fused kernel)
    gem::Sample2* d_samp_scene;    // samples in scene order (unfused kernels)
    int* d_samp_off;               // [n_scenes + 1] offsets into d_samp_scene
    int n_tasks;
    int task_tb, task_seg;     // tblock/segment the task list was built for
    // edge-list path
    void* graph;
    // reverse mode (k_adjoint.cu): checkpoints of the forward run
    void* adj;
    // persistent kernel: the items of one T-step block (an interior task, a
    // general task, or four narrow tasks: (kind, first task in d_ptasks)), the
    // items each must wait for (CSR), their completion counts, control words
    gem::Task* d_ptasks;
    int2* d_pitems;
    int* d_dep_off;
    int* d_dep_idx;
    unsigned* d_done;
    int n_pitems;
    // the items by warp class: interior items first, then general and narrow
    // ones, each in space order (the two queues of the persistent kernel)
    int* d_pq = nullptr;
    int n_pint = 0, n_pgen = 0;
    gem::DftItem* d_dft;           // every 2D cell-monitor accumulator
    std::vector<gem::TmzDev> h_scenes;   // host copy of d_scenes
    int n_dft;
    unsigned* d_ctl;
    int ctl_words;
    int* h_err;                  // pinned: copy of the sticky error word ctl[2] (cleared by fdtd_sync)
    long long spin_limit;        // polls a persistent-kernel wait makes before it gives up
    int opt_debug_skip;          // work item that never reports its first block done (-1 none)
    int opt_adj_store;           // FDTD_OPT_ADJ_STORE
    int opt_check_every;         // FDTD_OPT_CHECK_EVERY (0: off)
    int* d_bad;                  // sticky device word of the periodic finite check
    int* h_bad;                  // pinned copy of it (cleared by fdtd_sync)
    // CUDA graph of a step sequence
    int opt_graph;
    void* graph_exec;
    int64_t graph_t, graph_n;
    int graph_parity, graph_parity_after;
    int64_t graph_launches;
    cudaStream_t cap_stream;
};

namespace gem {
// kernels (k_tmz.cu)
int tmz_fused_launch(fdtd_ctx* c, int T, int warps, long long n0, int parity);
int tmz_naive_step(fdtd_ctx* c, long long n);
int dft_cells_launch(fdtd_ctx* c, const DftMon& m, long long n0, int nsteps);
int tmz_finite_check(fdtd_ctx* c, int* bad);
cudaError_t tmz_finite_launch(fdtd_ctx* c, int* d_flag);
int tmz_persistent_launch(fdtd_ctx* c, int T, long long n0, int n_blocks, int parity);
size_t tmz_fused_smem(int T, int warps, int V);   // V: 0 interior, 1 CPML, 2 lite
int tmz_design_band(fdtd_ctx* c, Scene2* s);
int tmz_design_coeffs(fdtd_ctx* c, Scene2* s, const double* eps_r, const double* sigma, size_t n, int* bad);
// raise a kernel's dynamic shared-memory limit to `bytes` on the current device,
// once (the attribute call is a driver round trip; later launches reuse it)
cudaError_t ensure_dyn_smem(const void* kernel, size_t bytes);
int dft_items_launch(fdtd_ctx* c, long long n0, int nsteps);
void adj_patch_descriptors(fdtd_ctx* c, TmzDev* dev);
}  // namespace gem

namespace gem {
// 3D Yee (k_yee3d.cu)
int fdtd_create3(const fdtd_grid* grid, double dx, double dt, double courant, const uint8_t* mat,
                 const fdtd_material* table, int n_mat, void* stream, fdtd_ctx** out);
void fdtd_destroy3(fdtd_ctx* c);
int fdtd_set_source3(fdtd_ctx* c, int kind, int i, int j, int k, int comp, const double* params,
                     const float* samples, int64_t n_samples);
int fdtd_add_probe3(fdtd_ctx* c, int i, int j, int k, int comp, int* id);
int fdtd_add_dft_monitor3(fdtd_ctx* c, const int32_t* cells, int n_cells, const double* freqs, int n_freq, int* id);
int fdtd_add_dft_plane3(fdtd_ctx* c, int k, int comp_mask, const double* freqs, int n_freq, int* id);
int fdtd_step3(fdtd_ctx* c, int64_t n);
int fdtd_read_probe3(fdtd_ctx* c, int id, float* out, int64_t n);
int fdtd_read_dft3(fdtd_ctx* c, int id, float* re, float* im);
int fdtd_get_field3(fdtd_ctx* c, int comp, float* out, int on_device);
int fdtd_set_field3(fdtd_ctx* c, int comp, const float* in, int on_device);
int fdtd_reset3(fdtd_ctx* c);
int fdtd_save_state3(fdtd_ctx* c, void* buf, size_t* bytes);
int fdtd_load_state3(fdtd_ctx* c, const void* buf, size_t bytes);
int fdtd_check_finite3(fdtd_ctx* c);
// literal edge-list path (k_graph.cu)
void graph_free(fdtd_ctx* c);
// a scene of the context is a y-slab sub-domain (fdtd_create_slab)
bool ctx_has_slab(const fdtd_ctx* c);
// reverse mode (k_adjoint.cu)
int adj_checkpoint_if_due(fdtd_ctx* c);
int adj_next_boundary(const fdtd_ctx* c, int64_t t);
void adj_free(fdtd_ctx* c);
// edge-weight reverse mode: the forward keeps the fields of the window one cell
// around each design rectangle after every step (the fused kernels in place,
// the unfused pair through adj_edge_record)
bool adj_edge_mode(const fdtd_ctx* c);
int adj_edge_record(fdtd_ctx* c, int steps_done);
}  // namespace gem

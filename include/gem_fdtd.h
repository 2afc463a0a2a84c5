/*
 * gem_fdtd.h -- C ABI of the GB300 (sm_103a) FDTD library.
 *
 * The library advances Maxwell's curl equations on a Yee grid with the leapfrog
 * scheme of "Solving Maxwell's Equations with Non-Trainable Graph Neural Network
 * Message Passing" (arXiv 2405.00814):
 *   layer 1 (H from curl E), eqs. (8)(9), Prop. 2 first message-passing step;
 *   layer 2 (E from curl H), eq. (7),      Prop. 2 second step,
 * with per-cell update coefficients Ca = A_-/A_+, Cb = dt/(A_+ eps),
 * A_-/+ = 1 -/+ sigma dt/(2 eps) (Sec. III-B, eq. (7)); Da = 1 and Db = dt/(mu0 d)
 * because the medium is non-magnetic outside the absorber (Sec. III-A).
 *
 * 2D runs are TMz (Ez, Hx, Hy): the paper's TE formulation (Ey, Hx, Hz in the
 * x-z plane, eqs. (3)-(5)) under the rotation x'=x, y'=z, z'=-y.  3D runs use
 * the six-component Yee cell the paper says follows directly (Sec. III-B).
 *
 * Grid conventions.  Cell (i, j[, k]) owns Ez(i, j) at (i dx, j dy), Hx(i, j) at
 * (i, j+1/2), Hy(i, j) at (i+1/2, j) (3D: Ex (i+1/2, j, k), Ey (i, j+1/2, k),
 * Ez (i, j, k+1/2), Hx (i, j+1/2, k+1/2), Hy (i+1/2, j, k+1/2), Hz (i+1/2, j+1/2, k)).
 * Host arrays are row-major with x fastest: [ny][nx] or [nz][ny][nx].
 * PEC walls sit at index 0 (stored zeros) and at index N (ghost zeros).
 * The absorber is a convolutional PML (Roden & Gedney) backed by that PEC; the
 * paper's own absorber is Berenger's split field (Sec. III-C, eqs. (10)-(13)).
 *
 * Ownership.  The library copies every input at call time and keeps no caller
 * pointer.  It owns all device memory of a context.  Output buffers are
 * allocated by the caller.  A context is not thread-safe; all of its work is
 * ordered on the CUDA stream given at creation (NULL = the legacy default
 * stream).  fdtd_step* only enqueue work; the fdtd_read_* and fdtd_get_* calls
 * synchronise the stream before they return.
 *
 * Errors.  Every int-returning call returns FDTD_OK (0) or a negative code;
 * fdtd_last_error() then returns a message owned by the context (valid until
 * the next call on it).  A call that fails leaves the simulation state as it
 * was, except FDTD_ECUDA, after which the context should be destroyed.
 */
#ifndef GEM_FDTD_H
#define GEM_FDTD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FDTD_OK 0
#define FDTD_EINVAL (-1)    /* bad argument (out-of-range index, size, kind...) */
#define FDTD_ENOMEM (-2)    /* device or host allocation failed */
#define FDTD_ECUDA (-3)     /* a CUDA call failed */
#define FDTD_EUNSTABLE (-4) /* dt above the Courant limit, or non-finite fields found */
#define FDTD_ETIMEOUT (-5)  /* a bounded device-side wait gave up */
#define FDTD_ESTATE (-6)    /* call not valid in the context's current state */

#define FDTD_PEC 0          /* plain PEC box */
#define FDTD_CPML 1         /* CPML of pml_cells cells on every face, backed by PEC */
#define FDTD_SPLIT_PML 2    /* 2D only: the paper's own absorber (Sec. III-C, eqs. (10)-(13)), Berenger's
                               split-field PML of pml_cells cells on every face, backed by PEC: Ez = Ezx + Ezy
                               in the layer, each part damped by the graded conductivity of its derivative's
                               axis, H by the matched sigma* = sigma mu0/eps0, semi-implicit as eq. (7);
                               sigma = sigma_max (depth/d)^3, sigma_max = 3.2 / (eta0 delta).  The layer's
                               cells must be vacuum (eps_r 1, sigma 0).  Steps with the temporally blocked
                               kernels (FDTD_OPT_KERNEL 0) or the unfused pair (1; also used in place of 2). */

/* field components */
#define FDTD_EX 0
#define FDTD_EY 1
#define FDTD_EZ 2
#define FDTD_HX 3
#define FDTD_HY 4
#define FDTD_HZ 5

/* source kinds (waveforms s(t) sampled at t = (n+1) dt after step n) */
#define FDTD_SRC_RICKER 0    /* params[0] = f_peak: (1-2a) e^{-a}, a = (pi f (t - 1.5/f))^2 */
#define FDTD_SRC_GAUSS_MOD 1 /* params[0] = f0: e^{-((t-t0)/tg)^2} sin(2 pi f0 (t-t0)), tg = 1/f0, t0 = 4 tg */
#define FDTD_SRC_GAUSS 2     /* params[0] = f_max: e^{-((t-t0)/tg)^2}, tg = 1/f_max, t0 = 4 tg */
#define FDTD_SRC_SAMPLED 3   /* samples[n] = s((n+1) dt), n < n_samples; 0 after */
#define FDTD_SRC_SINE 4      /* params[0] = f: sin(2 pi f t), switched on at t = 0 (Sec. V-A's sinusoidal source) */

/* options (fdtd_set_option) */
#define FDTD_OPT_KERNEL 0    /* 2D: 0 = fused temporally blocked stream, two kernels per T-step block (default);
                                1 = one H and one E launch per step;
                                2 = persistent: one cooperative launch runs many T-step blocks of every scene,
                                    warps pulling (block, work item) pairs in order from two shared counters, one
                                    for interior items and one for the rest (CPML, design, sources, probes), served
                                    by warps with 128 and 248 registers; an item waits (bounded) only for the items
                                    of the previous block whose regions meet its own, so there is no barrier between
                                    blocks (a context with a split-field PML steps with the unfused pair instead).
                                3D: 0 = fused z-marching kernel (default), 1 = one H and one E launch per step */
#define FDTD_OPT_TBLOCK 1    /* time steps per HBM pass of the fused kernel: 2D 1..4; 3D 1 or 2 (2, the 3D
                                default: the two-step z-marching kernel takes the steps in pairs, an odd last
                                step runs the one-step kernel; with more than 4 plane monitors every step does) */
#define FDTD_OPT_SEGMENT 2   /* 2D: rows per warp task of the fused kernel (>= 8);
                                3D: planes per z-segment of the fused z-marching kernels (>= 1; 0, the
                                default = 24 for the one-step kernel, 48 for the two-step one) */
#define FDTD_OPT_WARPS 3     /* warps per CTA of the fused kernel, 1..8 */
#define FDTD_OPT_GRAPH 4     /* 1: fdtd_step records its launches into a CUDA graph and replays it when called
                                again with the same start step, step count and buffer parity (e.g. after fdtd_reset) */
#define FDTD_OPT_SPIN_LIMIT 5     /* polls (about 0.1 us each) a persistent-kernel wait for another work item makes
                                     before it gives up */
#define FDTD_OPT_DEBUG_STALL_ITEM 6 /* test hook: in the next persistent launch only, the work item of this index
                                       (0 <= v < the launch's items per block) never reports its first block done, so
                                       the items that wait on it give up after FDTD_OPT_SPIN_LIMIT polls (-1 = off; reset
                                       to -1 by that launch); fdtd_sync then returns FDTD_ETIMEOUT.  The timeout is
                                       sticky: later persistent launches return without stepping until fdtd_sync has
                                       reported it */
#define FDTD_OPT_ADJ_STORE 7 /* reverse mode, read by fdtd_set_checkpointing: 1 (default) = the forward pass keeps
                                E^{n+1} - E^n over every design rectangle for every step in device memory
                                (steps x design cells x 4 B) and fdtd_adjoint_grad needs no recompute;
                                0 = keep field checkpoints only and recompute each segment (less memory);
                                2 = for fdtd_edge_grad: the forward keeps Ez, Hx, Hy of the window one
                                cell wider than each design rectangle after every step
                                (steps x (w + 2)(h + 2) x 12 B) */
#define FDTD_OPT_SEGMENT_B 8 /* 2D: rows per warp task of the boundary kernels (CPML slabs, source, probes, design,
                                ragged edge), forward and reverse sweep; 0 (default) = max(8, segment / 2).
                                Those warps carry a longer serial chain per row than interior ones */
#define FDTD_OPT_CHECK_EVERY 9 /* 2D: N > 0 = fdtd_step scans every field for NaN/Inf each time the step count
                                  passes a multiple of N (at the end of that T-step block; one extra launch over
                                  Ez, Hx, Hy), into a sticky device flag that fdtd_sync reports as FDTD_EUNSTABLE
                                  -- a blow-up found without synchronising the time loop; 0 (default) = off */
#define FDTD_OPT_TAPER 10    /* 2D, kernel 0: percent (0..60) of each strip's interior rows cut into tail
                                segments of half the FDTD_OPT_SEGMENT height; the interior list then runs
                                its CTAs tallest first (on the GPU, CTAs start in launch order), so the short
                                tasks fill the SMs the tall ones leave at the end of a T-step block.  0 (default)
                                = uniform segments in space order.  Results agree to FP32 rounding (other task
                                bounds move a few rows between the interior and the general kernels) */
#define FDTD_OPT_WARPS_B 11  /* 2D, kernels 0 and 2: warps per CTA of the CPML kernels of the forward step, 1..8
                                (default 2).  A CPML CTA holds 7 staged rows of 7 arrays per warp and about 220
                                registers per thread, so it leaves room for fewer interior CTAs on its SM; wider
                                CPML CTAs put the CPML warps on fewer SMs.  Results agree to FP32 rounding */
#define FDTD_OPT_PLAYOUT 12  /* 2D, kernel 2 (T 2..4, not in edge-weight mode): the persistent launch's CTAs.
                                0 (default) = one 12-warp CTA per SM, 8 interior warps at 128 registers and 4
                                general warps at 248; k >= 1 = one 16-warp CTA per SM, the first k (at most all
                                but one) running general and narrow items on 8 warps at 232 registers, every
                                other CTA 16 interior warps at 128.  Results agree to FP32 rounding */
#define FDTD_OPT_BULK 13     /* 2D, kernel 0: 1 = the interior kernel brings each row in with cp.async.bulk
                                copies (the TMA engine; one lane per row: Ez, Hx, Hy and the material window,
                                completing on a per-stage mbarrier) instead of 16-byte cp.async per lane; used
                                where every interior task's field rows start on 16 bytes.  Each mbarrier wait is
                                bounded by FDTD_OPT_SPIN_LIMIT polls, after which fdtd_sync reports
                                FDTD_ETIMEOUT.  0 (default) = cp.async.  Results are bit-identical */

typedef struct fdtd_ctx fdtd_ctx;

typedef struct {
    int dims;       /* 2 (TMz) or 3 */
    int nx, ny, nz; /* cells per axis (nz ignored for dims == 2); each >= 4 */
    int pml_cells;  /* absorbing layer depth in cells (FDTD_CPML, FDTD_SPLIT_PML) */
    int boundary;   /* FDTD_PEC, FDTD_CPML or FDTD_SPLIT_PML */
    double dy, dz;  /* cell sizes in m for y and z; <= 0 means "same as dx" */
} fdtd_grid;

typedef struct {
    double eps_r; /* relative permittivity, > 0 */
    double mu_r;  /* must be 1: the method assumes a non-magnetic medium (Sec. III-A) */
    double sigma; /* electric conductivity, S/m, >= 0 */
} fdtd_material;

/* Create a context for one scene (Sec. III-B: grid, dx, dt, material map).
 * dx: cell size in m (> 0).  dt: time step in s; if dt <= 0 the step is
 * courant * (Courant limit), courant in (0, 1].  A dt above the limit returns
 * FDTD_EUNSTABLE.  mat_idx: host uint8 map [ny][nx] (2D) or [nz][ny][nx] (3D) of
 * indices into table[0..n_mat-1]; 1 <= n_mat <= 255 (index 255 is reserved).
 * cuda_stream: a cudaStream_t or NULL.  *out receives the context. */
int fdtd_create(const fdtd_grid* grid, double dx, double dt, double courant, const uint8_t* mat_idx,
                const fdtd_material* table, int n_mat, void* cuda_stream, fdtd_ctx** out);

/* Create one context holding n_scenes independent 2D scenes of possibly
 * different sizes (the paper's many-simulation workloads, Sec. V-A); arrays
 * have one entry per scene.  fdtd_step advances every scene; per-scene calls act
 * on the scene chosen with fdtd_select_scene (scene 0 initially). */
int fdtd_create_batch(int n_scenes, const fdtd_grid* grids, const double* dx, const double* dt,
                      const uint8_t* const* mat_idx, const fdtd_material* const* tables,
                      const int* n_mat, void* cuda_stream, fdtd_ctx** out);
int fdtd_select_scene(fdtd_ctx* ctx, int scene);

/* y-slab sub-domain of a 2D grid: the domain decomposition the paper's related
 * work describes (Sec. II: the grid split into sub-domains, each advanced by its
 * own processing unit, the solutions combined), for grids larger than one GPU.
 * The context owns rows [j0, j1) of the whole grid `grid` (nx x ny, boundary
 * FDTD_PEC or FDTD_CPML) and holds `ghost` (1..64) extra rows on each side that
 * has a neighbour: local row r is grid row r + j0 - ghost_lo, where ghost_lo =
 * ghost if j0 > 0 else 0 (likewise ghost_hi above j1 < ny).  Every local-index
 * call (sources, probes, monitors, fields) uses those local rows.
 * mat_idx: host uint8 map of the local rows, [j1 - j0 + ghost_lo + ghost_hi][nx];
 * the CPML profile is the whole grid's, and only the grid's real walls are PEC.
 * Layer 1 reads Ez one row up and layer 2 reads Hx one row down (eqs. (7)-(9)),
 * so a step spoils one more ghost row at each cut: fdtd_step takes at most
 * `ghost` steps per call (FDTD_EINVAL otherwise), after which the caller must
 * refresh the ghost rows from the neighbours with fdtd_halo_export /
 * fdtd_halo_import before the next step.  A source cell within `ghost` rows of
 * a cut must be set in both slabs that hold it.  Requires j1 - j0 >= ghost.
 * Not available on a slab: design rectangles, reverse mode, the edge-list path
 * and graph export, autotuning, the split-field PML, batches. */
int fdtd_create_slab(const fdtd_grid* grid, int j0, int j1, int ghost, double dx, double dt, double courant,
                     const uint8_t* mat_idx, const fdtd_material* table, int n_mat, void* cuda_stream,
                     fdtd_ctx** out);
/* Floats in one side's halo: n_arrays x ghost x nx, n_arrays = 7 with a CPML
 * (Ez, Hx, Hy, psi_Ezx, psi_Ezy, psi_Hxy, psi_Hyx), 3 without; 0 if not a slab. */
int64_t fdtd_halo_count(const fdtd_ctx* ctx);
/* Copy the `ghost` owned rows next to a cut (side 0: rows j0 .. j0 + ghost - 1;
 * side 1: rows j1 - ghost .. j1 - 1) of every halo array, packed as
 * [array][row][nx] floats, into buf (host, or device when on_device != 0).
 * This is what the neighbour across that cut imports.  Ordered on the
 * context's stream; synchronises for a host buffer.  FDTD_EINVAL: not a slab,
 * side not 0/1, no neighbour on that side, NULL buf. */
int fdtd_halo_export(fdtd_ctx* ctx, int side, float* buf, int on_device);
/* Overwrite the ghost rows below the slab (side 0) or above it (side 1) from a
 * buffer the neighbour exported from its opposite side (the rows land in this
 * context's own memory; the library reads no other context's memory).  Ordered
 * on this context's stream: when the neighbour uses another stream, order its
 * export before this import (an event, or a synchronise).  Same errors. */
int fdtd_halo_import(fdtd_ctx* ctx, int side, const float* buf, int on_device);
/* Owned rows [*j0, *j1) of the whole grid and the grid row of local row 0
 * (0, ny, 0 for a whole grid).  NULL outputs are skipped. */
int fdtd_slab_rows(const fdtd_ctx* ctx, int* j0, int* j1, int* row_offset);
int fdtd_num_scenes(const fdtd_ctx* ctx);

void fdtd_destroy(fdtd_ctx* ctx);
const char* fdtd_last_error(const fdtd_ctx* ctx);
int fdtd_set_option(fdtd_ctx* ctx, int option, int64_t value);
int64_t fdtd_get_option(const fdtd_ctx* ctx, int option);

/* Soft (additive) point source of the selected scene: after the E update of
 * step n the component at (i, j[, k]) gets s((n+1) dt) added (Sec. V-A: sources
 * at random positions; Sec. V-B: point sources).  2D accepts FDTD_EZ only, at
 * 1 <= i < nx, 1 <= j < ny.  params: one double per kind (see FDTD_SRC_*);
 * samples/n_samples for FDTD_SRC_SAMPLED (copied).  Replaces any earlier source. */
int fdtd_set_source(fdtd_ctx* ctx, int kind, int i, int j, int k, int component, const double* params,
                    const float* samples, int64_t n_samples);

/* 2D only: a line source -- every cell (i, j) with j0 <= j < j1 of column i gets
 * the same waveform added to Ez after each E update, as the photonic-crystal
 * example excites every cell across its waveguide (Sec. V-B).  Same kinds and
 * arguments as fdtd_set_source; 1 <= i < nx, 1 <= j0 < j1 <= ny.  Replaces any
 * earlier source (a point source is the line j1 = j0 + 1). */
int fdtd_set_line_source(fdtd_ctx* ctx, int kind, int i, int j0, int j1, const double* params, const float* samples,
                         int64_t n_samples);

/* Replace the material map and table of the selected 2D scene in place (same
 * grid, boundary, dt), to solve a new geometry in an existing context without
 * re-creating it.  mat_idx: [ny][nx] indices into table, host memory; table:
 * n_mat (1..255) entries checked as for fdtd_create; eq. (7) gives the new
 * coefficients.  The map is copied on the context's stream (asynchronously when
 * mat_idx is page-locked: keep it unchanged until the next call that
 * synchronises); its indices are not scanned, and a cell whose index is >= n_mat
 * takes zero coefficients, i.e. acts as a PEC cell.  The walls i = 0 and j = 0
 * stay PEC.  Fields, source, probes and monitors are kept (fdtd_reset starts a
 * new solve); a design rectangle keeps its own values; a recorded CUDA graph
 * stays valid.  FDTD_EINVAL: NULL pointers, n_mat outside 1..255, a rejected
 * table entry, a non-vacuum cell in a split-field PML layer, a 3D context. */
int fdtd_set_materials(fdtd_ctx* ctx, const uint8_t* mat_idx, const fdtd_material* table, int n_mat);

/* Continuous permittivity over a rectangle of the selected 2D scene -- the
 * design region of inverse design, where every cell has its own eps_r.  Cells
 * [i0, i0+w) x [j0, j0+h) take eps_r[dj*w + di] and sigma[dj*w + di] (sigma NULL
 * = 0) instead of their material-table entry; coefficients follow eq. (7).
 * eps_r and sigma are host arrays, or device arrays when on_device != 0 (then
 * the coefficients are formed by a kernel and no value crosses to the host).
 * The rectangle must avoid the PEC walls: 1 <= i0, i0 + w <= nx, same for j.
 * Calling it again replaces the values (same rectangle) or the rectangle; while
 * checkpointing is on (fdtd_set_checkpointing) the rectangle may move but not
 * change its size (FDTD_EINVAL).  Synchronises.  FDTD_EINVAL also for an
 * eps_r <= 0 or sigma < 0 (found on the device for device arrays, after which
 * the scene has no design rectangle). */
int fdtd_set_design(fdtd_ctx* ctx, int i0, int j0, int w, int h, const double* eps_r, const double* sigma,
                    int on_device);

/* Probe: records the component at (i, j[, k]) after every following step
 * (after the source) -- the waveforms of Fig. 2d.  *probe_id gets its index.
 * Probes must be added before the first step after a reset. */
int fdtd_add_probe(fdtd_ctx* ctx, int i, int j, int k, int component, int* probe_id);

/* Running DFT of Ez at cells: F(f) = sum_{n>=1} Ez^n exp(-i 2 pi f n dt) dt over
 * all steps taken after the monitor was added (frequency-domain responses via a
 * Fourier transform of sampled waveforms, Sec. I).  cells: n_cells (i, j) pairs
 * (2D) or (i, j, k) triples (3D).  Accumulated in compensated (Kahan) FP32. */
int fdtd_add_dft_monitor(fdtd_ctx* ctx, const int32_t* cells, int n_cells, const double* freqs_hz,
                         int n_freq, int* mon_id);

/* 3D only: running DFT of the E components in comp_mask (bit c = FDTD_EX+c) over
 * the whole plane z = k (cell index k), same convention as above; 1..16
 * frequencies (FDTD_EINVAL otherwise). */
int fdtd_add_dft_plane(fdtd_ctx* ctx, int k, int comp_mask, const double* freqs_hz, int n_freq,
                       int* mon_id);

/* Advance every scene n_steps leapfrog steps with the implicit-stencil kernels
 * (layers 1 and 2 fused, temporally blocked; FDTD_OPT_KERNEL selects the
 * unfused pair).  Asynchronous. */
int fdtd_step(fdtd_ctx* ctx, int64_t n_steps);

/* Same recurrence computed literally as the paper's two message-passing layers
 * over an explicit edge list (Prop. 1 numbering, Prop. 2 layers): per step one
 * sparse gather per layer, h_l = sum_{l_n in N(v_l)} w_{l,l_n} h_{l_n}.  2D only. */
int fdtd_step_edgelist(fdtd_ctx* ctx, int64_t n_steps);

/* Export layer 1 or 2 of that graph (selected scene): *n_nodes and *n_edges are
 * always written; src/dst/w (n_edges entries each, caller-allocated, host) are
 * filled when non-NULL.  Edges are grouped by destination; rows of nodes the
 * layer does not update carry one self edge of weight 1.  Node numbering:
 * Prop. 1 with k -> j (u = i + 3 j nx for Hx, q = 2 i + nx(3 j + 1) for Hy,
 * t = 2 i + 1 + nx(3 j + 1) for Ez), then CPML auxiliary nodes. */
int fdtd_export_graph(fdtd_ctx* ctx, int layer, int64_t* n_nodes, int64_t* n_edges, int32_t* src,
                      int32_t* dst, float* w);

/* Copy out n values of a probe (n <= steps recorded).  Synchronises. */
int fdtd_read_probe(fdtd_ctx* ctx, int probe_id, float* out, int64_t n);

/* Copy out a DFT monitor: re/im [n_cells][n_freq] (cell monitor) or
 * [n_comp][n_freq][ny][nx] (plane monitor).  Synchronises. */
int fdtd_read_dft(fdtd_ctx* ctx, int mon_id, float* re, float* im);

/* Copy a field component of the selected scene to out ([ny][nx] or [nz][ny][nx]
 * floats); on_device != 0 means out is a device pointer.  Synchronises. */
int fdtd_get_field(fdtd_ctx* ctx, int component, float* out, int on_device);
/* Overwrite a field component from in (same layout). */
int fdtd_set_field(fdtd_ctx* ctx, int component, const float* in, int on_device);

/* Zero every field, auxiliary, probe record and DFT accumulator; time -> 0. */
int fdtd_reset(fdtd_ctx* ctx);
/* Steps taken since creation or the last reset. */
int64_t fdtd_time_step(const fdtd_ctx* ctx);
/* Kernel launches issued by this context so far (all kinds). */
int64_t fdtd_launch_count(const fdtd_ctx* ctx);

/* Checkpoint: the full state (fields, CPML auxiliaries, DFT accumulators, time)
 * of every scene.  buf == NULL: *bytes receives the size needed.  Otherwise
 * *bytes is the buffer's size on input and the bytes written on output; the
 * buffer is host memory.  fdtd_load_state restores a buffer from the same
 * context configuration. */
int fdtd_save_state(fdtd_ctx* ctx, void* buf, size_t* bytes);
int fdtd_load_state(fdtd_ctx* ctx, const void* buf, size_t bytes);

/* Wait for the context's stream.  Returns FDTD_ETIMEOUT if a bounded device
 * wait (the persistent kernel's wait for another work item) gave up since the last call: the
 * kernel then stopped early, the context stays usable, and the fields hold the
 * state of an incomplete step sequence.  Otherwise returns FDTD_EUNSTABLE if the
 * periodic finite check (FDTD_OPT_CHECK_EVERY) found a non-finite value since
 * the last call.  Each condition is reported once, then cleared. */
int fdtd_sync(fdtd_ctx* ctx);

/* Pick the 2D kernel options for the current scenes (one large scene, or a
 * batch: Sec. V-A runs many simulations of varying size): time every candidate
 * of (kernel 0: T 2..4, segment 16..96 in steps of 4, warps 2, 4 or 8, CPML
 * warps (FDTD_OPT_WARPS_B) 2, 4 or 8; kernel 2, not for a split-field PML:
 * T 2..4, segment 32, 64, 96 or 128, FDTD_OPT_PLAYOUT 0, 24, 48 or 64) for
 * trial_steps steps, time the four fastest twice more for 4 x trial_steps, keep
 * the best; then, for kernel 0, search the segment height (-8..+8 rows around
 * the candidate's, in steps of 4) and FDTD_OPT_SEGMENT_B (automatic, 4..32 in
 * steps of 4) jointly around the two best (T, warps, CPML warps) settings of
 * the first pass, then FDTD_OPT_TAPER 10, 20, 30, 45 with the segment height
 * raised by 0, 8, 16 or 24 rows (each kept only if 1 % faster).  Leaves the
 * context reset (t = 0, zero fields).  *best_ms gets the best time per step. */
int fdtd_autotune(fdtd_ctx* ctx, int trial_steps, double* best_ms);

/* Returns FDTD_EUNSTABLE if any field of any scene is not finite. Synchronises. */
int fdtd_check_finite(fdtd_ctx* ctx);

/* Reverse mode (2D).  The paper notes that message-passing layers are
 * differentiable (Sec. IV-A); these calls compute the discrete adjoint of the
 * two layers of Prop. 2 -- the transposed layers in reverse time order.
 *
 * fdtd_set_checkpointing: from now on, fdtd_step works in segments of `every`
 * steps (0 turns reverse mode off and frees its memory).  With FDTD_OPT_ADJ_STORE
 * = 1 it records r^n = E^{n+1} - E^n (before the source) over every design
 * rectangle for every step, one device block per segment; with 0 it saves the
 * full state of every scene (fields and CPML auxiliaries) at each segment start
 * instead.  All of it lives in device memory owned by the context. */
int fdtd_set_checkpointing(fdtd_ctx* ctx, int every);

/* Gradient of a real loss L(F) of the running DFTs with respect to eps_r over
 * every scene's design rectangle (fdtd_set_design), after a forward run of N
 * steps from reset with checkpointing on.  dLdF_re/dLdF_im: dL/dRe F and dL/dIm F
 * for every cell DFT monitor in creation order, [n_cells][n_freq] each,
 * concatenated (host).  The adjoint source at a monitor cell for step n is
 * sum_f (dL/dRe F cos(2 pi f (n+1) dt) - dL/dIm F sin(2 pi f (n+1) dt)) dt.
 * Segments are reversed newest first (in checkpoint mode each is first
 * recomputed from its checkpoint to record r^n).  With e^{n+1} = dL/dE^{n+1},
 *   dL/deps_r = sum_n e^{n+1} (dCa/deps_r E^n + dCb/deps_r curlH^{n+1/2})
 *             = -eps0 / (eps0 eps_r + sigma dt / 2) * sum_n e^{n+1} r^n,
 * since dCa/deps_r = -sigma dCb/deps_r and Cb curlH = E^{n+1} - Ca E^n.  grad
 * receives dL/deps_r as [scene][h][w] floats (host, or device when on_device !=
 * 0).  The fields are left in an unspecified state: call fdtd_reset before the
 * next forward run. */
int fdtd_adjoint_grad(fdtd_ctx* ctx, const float* dLdF_re, const float* dLdF_im, float* grad, int on_device);

/* Learnable edge weights.  The paper's layers have fixed weights read off the
 * update equations, and it notes that message-passing layers are differentiable
 * (Sec. IV-A); this is the gradient of the same loss as fdtd_adjoint_grad with
 * respect to each weight of the graph of Prop. 1 whose destination node belongs
 * to a design cell (i, j), treating every weight as an independent parameter.
 * A cell owns FDTD_EDGE_CLASSES weights, in this order (destination <- source,
 * TMz names, the weight's physical value in brackets, eqs. (7)-(9)):
 *   layer 2:  0 Ez(i,j) <- Ez(i,j) [Ca]       1 Ez(i,j) <- Hy(i,j) [Cb/dx]
 *             2 Ez(i,j) <- Hy(i-1,j) [-Cb/dx] 3 Ez(i,j) <- Hx(i,j) [-Cb/dy]
 *             4 Ez(i,j) <- Hx(i,j-1) [Cb/dy]
 *   layer 1:  5 Hx(i,j) <- Hx(i,j) [1]        6 Hx(i,j) <- Ez(i,j+1) [-Db/dy]
 *             7 Hx(i,j) <- Ez(i,j) [Db/dy]    8 Hy(i,j) <- Hy(i,j) [1]
 *             9 Hy(i,j) <- Ez(i+1,j) [Db/dx] 10 Hy(i,j) <- Ez(i,j) [-Db/dx]
 * with Db = dt / mu0.  dL/dw = sum over steps n of (dL/d destination after the
 * layer) x (source before the layer): dL/dE^{n+1} x (E^n or H^{n+1/2}) for layer 2,
 * dL/dH^{n+1/2} x (E^n or H^{n-1/2}) for layer 1.
 * Needs a forward run of N >= 1 steps from reset with FDTD_OPT_ADJ_STORE = 2 set
 * before fdtd_set_checkpointing (FDTD_ESTATE otherwise), every scene with a
 * design rectangle whose one-cell ring lies outside the CPML and inside the grid
 * (the forward returns FDTD_EINVAL at its first step otherwise).  dLdF_re,
 * dLdF_im: as for fdtd_adjoint_grad.  grad receives [scene][FDTD_EDGE_CLASSES][h][w]
 * floats (host, or device when on_device != 0).  The fields are left in an
 * unspecified state: call fdtd_reset before the next forward run. */
#define FDTD_EDGE_CLASSES 11
int fdtd_edge_grad(fdtd_ctx* ctx, const float* dLdF_re, const float* dLdF_im, float* grad, int on_device);

/* Largest graph fdtd_mp_steps_noalloc accepts (nodes). */
#define FDTD_MP_NOALLOC_MAX_NODES (1 << 22)

/* Allocation-free message passing.  The paper has no counterpart to this
 * entry point; it exists for callers that cannot allocate device memory -- a
 * host application whose own allocator owns all device memory and allows no
 * allocation behind its back, or a real-time loop that cannot absorb the
 * device-wide synchronisation of cudaMalloc/cudaFree.  It runs n_steps applications of h <- W2 (W1 h) for two
 * layers given as CSR by destination (rowptr[n_nodes + 1], col and w per edge,
 * as fdtd_export_graph lists them after sorting by destination), with every
 * pointer a caller-allocated device pointer; h (n_nodes floats) is read and
 * overwritten.  No soft source is applied.  The state between the layers lives
 * in a fixed device array of FDTD_MP_NOALLOC_MAX_NODES floats (16 MiB) that
 * every GPU loading the library keeps until the process exits; it never calls
 * cudaMalloc, cudaFree or any allocating routine.  The first call on a device
 * looks that array's address up (cudaGetSymbolAddress with the device
 * current), so make the first call before any stream capture begins.  The
 * address is kept for the life of the device's primary context: after
 * cudaDeviceReset (or anything else that destroys that context) in this
 * process, do not call this entry point again.  All calls share the array: calls that overlap on the GPU (different streams, or
 * different host threads on one device) race and corrupt each other's results.
 * Returns FDTD_EINVAL for NULL pointers, n_nodes < 1 or n_nodes larger than
 * FDTD_MP_NOALLOC_MAX_NODES, n_steps < 0; FDTD_ECUDA if a launch fails.
 * Work is enqueued on cuda_stream (NULL = legacy default stream); the call
 * does not synchronise. */
int fdtd_mp_steps_noalloc(const int32_t* rowptr1, const int32_t* col1, const float* w1, const int32_t* rowptr2,
                          const int32_t* col2, const float* w2, float* h, int64_t n_nodes, int64_t n_steps,
                          void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GEM_FDTD_H */

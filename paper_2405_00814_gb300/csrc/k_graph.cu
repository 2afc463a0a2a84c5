// Literal message-passing form of the leapfrog step (Prop. 1 and Prop. 2).
//
// The graph G(V, E) of Prop. 1 is built explicitly on the host: 3 nodes per
// cell, numbered u(i,j) = i + 3 j nx (Hx), q(i,j) = 2 i + nx (3 j + 1) (Hy),
// t(i,j) = 2 i + 1 + nx (3 j + 1) (Ez) -- the paper's TE numbering with k -> j in
// the TMz rotation -- followed by one node per CPML auxiliary psi.  Each of the
// two layers of Prop. 2 is a sparse matrix stored by destination (CSR): row v
// lists N(v) and the static weights w_{v, v_n} read off eqs. (7)-(9); nodes a
// layer does not update keep a single self edge of weight 1 (Prop. 2: neurons
// updated earlier remain constant).  One step is h <- W2 (W1 h), one gather
// kernel per layer, then the soft source.  The neighbourhood offsets follow the
// update equations: E gathers from H at (i, j), (i-1, j), (i, j-1); H gathers
// from E at (i, j), (i+1, j), (i, j+1).
//
// A scene with the split-field PML (Sec. III-C) uses the paper's graph with
// absorbing boundaries instead (Sec. IV-B): 4 nodes per cell, u(i,j) = i + 4 j nx
// (Hx), q(i,j) = 3 i + nx (4 j + 1) (Hy), tx = q + 1 (Ezx), tz = q + 2 (Ezy); Ezx
// gathers Hy at (i, j), (i-1, j), Ezy gathers Hx at (i, j), (i, j-1), and H gathers
// both E parts at the forward neighbours.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "gem_internal.h"

namespace gem {

namespace {
const double kC0g = 299792458.0;
const double kMu0g = 4.0e-7 * M_PI;
const double kEps0g = 1.0 / (kMu0g * kC0g * kC0g);
}  // namespace

struct SceneGraph {
    int64_t n_nodes;
    int64_t nnz[2];
    int* d_rowptr[2];
    int* d_col[2];
    float* d_w[2];
    float* d_h[2];          // node state ping-pong
    int n_psi;
    int* d_psi;             // per psi node: (type << 29) | storage-free cell index j * nx + i
    int64_t psi_base;
    int split;              // 4-node graph of the split-field layer
};

struct Graph {
    std::vector<SceneGraph> g;
};

static inline int64_t node_t(int nx, int i, int j) { return 2 * (int64_t)i + 1 + (int64_t)nx * (3 * (int64_t)j + 1); }
static inline int64_t node_u(int nx, int i, int j) { return (int64_t)i + 3 * (int64_t)j * nx; }
static inline int64_t node_q(int nx, int i, int j) { return 2 * (int64_t)i + (int64_t)nx * (3 * (int64_t)j + 1); }
// split-field graph (Sec. IV-B): kind 0 u (Hx), 1 q (Hy), 2 tx (Ezx), 3 tz (Ezy)
static inline int64_t node4(int nx, int kind, int i, int j) {
    if (kind == 0) return (int64_t)i + 4 * (int64_t)j * nx;
    return 3 * (int64_t)i + (kind - 1) + (int64_t)nx * (4 * (int64_t)j + 1);
}

// host copies of the FP32 profiles and coefficients the kernels use
struct HostScene {
    int nx, ny, pitch, rows;
    std::vector<float> prof;
    std::vector<float4> coef;
    std::vector<uint8_t> mat;      // padded
    std::vector<float4> dsg;
    float dbx, dby;
    int npml, split;
    int dsg_i0, dsg_j0, dsg_w, dsg_h;
};

static int fetch(fdtd_ctx* c, const Scene2* s, HostScene& h) {
    h.nx = s->nx; h.ny = s->ny; h.pitch = s->pitch; h.rows = s->rows;
    h.prof.resize(4 * (size_t)s->pitch + 4 * (size_t)s->rows);
    h.coef.resize(256);
    h.mat.resize((size_t)s->pitch * s->rows);
    cudaMemcpyAsync(h.prof.data(), s->d_prof, h.prof.size() * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(h.coef.data(), s->d_coef, 256 * sizeof(float4), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(h.mat.data(), s->d_mat, h.mat.size(), cudaMemcpyDeviceToHost, c->stream);
    if (s->d_dsg) {
        h.dsg.resize((size_t)s->dsg_w * s->dsg_h);
        cudaMemcpyAsync(h.dsg.data(), s->d_dsg, h.dsg.size() * sizeof(float4), cudaMemcpyDeviceToHost, c->stream);
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("graph: fetch scene: ") + cudaGetErrorString(e);
        return FDTD_ECUDA;
    }
    h.dbx = (float)(s->dt / (kMu0g * s->dx));
    h.dby = (float)(s->dt / (kMu0g * s->dy));
    h.npml = s->npml;
    h.split = s->split;
    h.dsg_i0 = s->dsg_i0; h.dsg_j0 = s->dsg_j0; h.dsg_w = s->d_dsg ? s->dsg_w : 0; h.dsg_h = s->dsg_h;
    return FDTD_OK;
}

// the two layers of the split-field graph, rows in node order, weights from
// the same FP32 profiles and coefficients the stencil kernels use
static void build_layer_split(const HostScene& h, int layer, std::vector<int>& rowptr, std::vector<int>& col,
                              std::vector<float>& w) {
    const int nx = h.nx, ny = h.ny, np = h.npml;
    const int64_t n_nodes = 4 * (int64_t)nx * ny;
    const float* px = h.prof.data();
    const float* py = h.prof.data() + 4 * h.pitch;
    rowptr.assign(n_nodes + 1, 0);
    col.clear();
    w.clear();
    col.reserve(n_nodes * 3);
    w.reserve(n_nodes * 3);
    auto put = [&](int64_t c, float v) {
        col.push_back((int)c);
        w.push_back(v);
    };
    for (int64_t v = 0; v < n_nodes; v++) {
        rowptr[v] = (int)col.size();
        const int j = (int)(v / (4 * (int64_t)nx));
        const int64_t r = v % (4 * (int64_t)nx);
        const int kind = r < nx ? 0 : 1 + (int)((r - nx) % 3);
        const int i = r < nx ? (int)r : (int)((r - nx) / 3);
        if (layer == 1 && kind == 0) {                 // Hx(i,j)
            const bool ly = j < np || j >= ny - np;
            const float da = ly ? py[2 * h.rows + j + PAD_Y] : 1.f, db = ly ? py[3 * h.rows + j + PAD_Y] : h.dby;
            put(v, da);
            if (j + 1 < ny) {
                put(node4(nx, 2, i, j + 1), -db);
                put(node4(nx, 3, i, j + 1), -db);
            }
            put(node4(nx, 2, i, j), db);
            put(node4(nx, 3, i, j), db);
        } else if (layer == 1 && kind == 1) {          // Hy(i,j)
            const bool lx = i < np || i >= nx - np;
            const float da = lx ? px[2 * h.pitch + i + PAD_X] : 1.f, db = lx ? px[3 * h.pitch + i + PAD_X] : h.dbx;
            put(v, da);
            if (i + 1 < nx) {
                put(node4(nx, 2, i + 1, j), db);
                put(node4(nx, 3, i + 1, j), db);
            }
            put(node4(nx, 2, i, j), -db);
            put(node4(nx, 3, i, j), -db);
        } else if (layer == 2 && kind >= 2 && i >= 1 && j >= 1) {
            float4 co = h.coef[h.mat[(size_t)(j + PAD_Y) * h.pitch + i + PAD_X]];
            const int di = i - h.dsg_i0, dj = j - h.dsg_j0;
            if (h.dsg_w > 0 && di >= 0 && di < h.dsg_w && dj >= 0 && dj < h.dsg_h) co = h.dsg[(size_t)dj * h.dsg_w + di];
            const bool lx = i < np || i > nx - np, ly = j < np || j > ny - np;
            if (kind == 2) {                           // Ezx(i,j)
                const float a = lx ? px[i + PAD_X] : co.x, b = lx ? px[h.pitch + i + PAD_X] : co.y;
                put(v, a);
                put(node4(nx, 1, i, j), b);
                put(node4(nx, 1, i - 1, j), -b);
            } else {                                   // Ezy(i,j)
                const float a = ly ? py[j + PAD_Y] : co.x, b = ly ? py[h.rows + j + PAD_Y] : co.z;
                put(v, a);
                put(node4(nx, 0, i, j), -b);
                put(node4(nx, 0, i, j - 1), b);
            }
        } else {
            put(v, 1.f);                               // not updated by this layer
        }
    }
    rowptr[n_nodes] = (int)col.size();
}

// psi node lists: type 0 psi_Hxy, 1 psi_Hyx, 2 psi_Ezx, 3 psi_Ezy (same storage slots F_PHXY, F_PHYX, F_PEZX, F_PEZY)
static void psi_lists(const HostScene& h, std::vector<int>& psi, std::vector<int64_t>& idx4) {
    const int nx = h.nx, ny = h.ny;
    const float* px = h.prof.data();
    const float* py = h.prof.data() + 4 * h.pitch;
    auto bEx = [&](int i) { return px[i + PAD_X]; };
    auto cEx = [&](int i) { return px[h.pitch + i + PAD_X]; };
    auto bHx = [&](int i) { return px[2 * h.pitch + i + PAD_X]; };
    auto cHx = [&](int i) { return px[3 * h.pitch + i + PAD_X]; };
    auto bEy = [&](int j) { return py[j + PAD_Y]; };
    auto cEy = [&](int j) { return py[h.rows + j + PAD_Y]; };
    auto bHy = [&](int j) { return py[2 * h.rows + j + PAD_Y]; };
    auto cHy = [&](int j) { return py[3 * h.rows + j + PAD_Y]; };
    const int64_t ncell = (int64_t)nx * ny;
    idx4.assign(4 * ncell, -1);
    const int64_t base = 3 * ncell;
    for (int type = 0; type < 4; type++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                bool has;
                if (type == 0) has = bHy(j) != 0.f || cHy(j) != 0.f;
                else if (type == 1) has = bHx(i) != 0.f || cHx(i) != 0.f;
                else if (type == 2) has = i >= 1 && j >= 1 && (bEx(i) != 0.f || cEx(i) != 0.f);
                else has = i >= 1 && j >= 1 && (bEy(j) != 0.f || cEy(j) != 0.f);
                if (!has) continue;
                idx4[type * ncell + (int64_t)j * nx + i] = base + (int64_t)psi.size();
                psi.push_back((type << 29) | (j * nx + i));
            }
}

// rows of one layer, in node order
static void build_layer(const HostScene& h, int layer, const std::vector<int>& psi, const std::vector<int64_t>& idx4,
                        std::vector<int>& rowptr, std::vector<int>& col, std::vector<float>& w) {
    const int nx = h.nx, ny = h.ny;
    const int64_t ncell = (int64_t)nx * ny;
    const int64_t n_nodes = 3 * ncell + (int64_t)psi.size();
    const float* px = h.prof.data();
    const float* py = h.prof.data() + 4 * h.pitch;
    rowptr.assign(n_nodes + 1, 0);
    col.clear();
    w.clear();
    col.reserve(n_nodes * 3);
    w.reserve(n_nodes * 3);
    auto put = [&](int64_t c, float v) {
        col.push_back((int)c);
        w.push_back(v);
    };
    for (int64_t v = 0; v < n_nodes; v++) {
        rowptr[v] = (int)col.size();
        if (v < 3 * ncell) {
            const int j = (int)(v / (3 * (int64_t)nx));
            const int64_t r = v % (3 * (int64_t)nx);
            int kind, i;   // 0 t (Ez), 1 u (Hx), 2 q (Hy)
            if (r < nx) {
                kind = 1;
                i = (int)r;
            } else {
                kind = ((r - nx) % 2 == 0) ? 2 : 0;
                i = (int)((r - nx) / 2);
            }
            const int64_t cell = (int64_t)j * nx + i;
            if (layer == 1 && kind == 1) {
                const float b = py[2 * h.rows + j + PAD_Y], cc = py[3 * h.rows + j + PAD_Y];
                const float a = h.dby * (1.f + cc);
                put(v, 1.f);
                if (j + 1 < ny) put(node_t(nx, i, j + 1), -a);
                put(node_t(nx, i, j), a);
                if (idx4[0 * ncell + cell] >= 0) put(idx4[0 * ncell + cell], -h.dby * b);
            } else if (layer == 1 && kind == 2) {
                const float b = px[2 * h.pitch + i + PAD_X], cc = px[3 * h.pitch + i + PAD_X];
                const float a = h.dbx * (1.f + cc);
                put(v, 1.f);
                if (i + 1 < nx) put(node_t(nx, i + 1, j), a);
                put(node_t(nx, i, j), -a);
                if (idx4[1 * ncell + cell] >= 0) put(idx4[1 * ncell + cell], h.dbx * b);
            } else if (layer == 2 && kind == 0 && i >= 1 && j >= 1) {
                const float4 co = h.coef[h.mat[(size_t)(j + PAD_Y) * h.pitch + i + PAD_X]];
                const float bx = px[i + PAD_X], cx = px[h.pitch + i + PAD_X];
                const float by = py[j + PAD_Y], cy = py[h.rows + j + PAD_Y];
                const float ax = co.y * (1.f + cx), ay = co.z * (1.f + cy);
                put(v, co.x);
                put(node_q(nx, i, j), ax);
                put(node_q(nx, i - 1, j), -ax);
                put(node_u(nx, i, j), -ay);
                put(node_u(nx, i, j - 1), ay);
                if (idx4[2 * ncell + cell] >= 0) put(idx4[2 * ncell + cell], co.y * bx);
                if (idx4[3 * ncell + cell] >= 0) put(idx4[3 * ncell + cell], -co.z * by);
            } else {
                put(v, 1.f);
            }
        } else {
            const int p = psi[v - 3 * ncell];
            const int type = p >> 29;
            const int cell = p & ((1 << 29) - 1);
            const int i = cell % nx, j = cell / nx;
            if (layer == 1 && type == 0) {
                const float b = py[2 * h.rows + j + PAD_Y], cc = py[3 * h.rows + j + PAD_Y];
                put(v, b);
                if (j + 1 < ny) put(node_t(nx, i, j + 1), cc);
                put(node_t(nx, i, j), -cc);
            } else if (layer == 1 && type == 1) {
                const float b = px[2 * h.pitch + i + PAD_X], cc = px[3 * h.pitch + i + PAD_X];
                put(v, b);
                if (i + 1 < nx) put(node_t(nx, i + 1, j), cc);
                put(node_t(nx, i, j), -cc);
            } else if (layer == 2 && type == 2) {
                const float b = px[i + PAD_X], cc = px[h.pitch + i + PAD_X];
                put(v, b);
                put(node_q(nx, i, j), cc);
                put(node_q(nx, i - 1, j), -cc);
            } else if (layer == 2 && type == 3) {
                const float b = py[j + PAD_Y], cc = py[h.rows + j + PAD_Y];
                put(v, b);
                put(node_u(nx, i, j), cc);
                put(node_u(nx, i, j - 1), -cc);
            } else {
                put(v, 1.f);
            }
        }
    }
    rowptr[n_nodes] = (int)col.size();
}

// design-rectangle cells take their own coefficients: patch the Ez rows
static void apply_design(const HostScene& h, const Scene2* s, std::vector<int>& rowptr, std::vector<int>& col,
                         std::vector<float>& w, const std::vector<int64_t>& idx4) {
    if (h.dsg.empty()) return;
    const int nx = h.nx;
    const int64_t ncell = (int64_t)nx * h.ny;
    const float* px = h.prof.data();
    const float* py = h.prof.data() + 4 * h.pitch;
    for (int dj = 0; dj < s->dsg_h; dj++)
        for (int di = 0; di < s->dsg_w; di++) {
            const int i = s->dsg_i0 + di, j = s->dsg_j0 + dj;
            const float4 co = h.dsg[(size_t)dj * s->dsg_w + di];
            const int64_t v = node_t(nx, i, j);
            int e = rowptr[v];
            const float cx = px[h.pitch + i + PAD_X], cy = py[h.rows + j + PAD_Y];
            const float ax = co.y * (1.f + cx), ay = co.z * (1.f + cy);
            w[e++] = co.x;
            w[e++] = ax;
            w[e++] = -ax;
            w[e++] = -ay;
            w[e++] = ay;
            const int64_t cell = (int64_t)j * nx + i;
            if (idx4[2 * ncell + cell] >= 0) w[e++] = co.y * px[i + PAD_X];
            if (idx4[3 * ncell + cell] >= 0) w[e++] = -co.z * py[j + PAD_Y];
            (void)col;
        }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
__global__ void k_mp_layer(const int* __restrict__ rowptr, const int* __restrict__ col, const float* __restrict__ w,
                           const float* __restrict__ x, float* __restrict__ y, int64_t n) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float acc = 0.f;
    const int e1 = rowptr[r + 1];
    for (int e = rowptr[r]; e < e1; e++) acc += w[e] * x[col[e]];
    y[r] = acc;
}

__device__ __forceinline__ size_t gsidx(int pitch, int i, int j) {
    return (size_t)(j + PAD_Y) * (size_t)pitch + (size_t)(i + PAD_X);
}

// fields <-> node vector (dir 0: fields to nodes, 1: nodes to fields)
__global__ void k_cells_nodes(const TmzDev* __restrict__ sc, int scene, int parity, float* h, int dir) {
    const TmzDev& S = sc[scene];
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (int64_t)S.nx * S.ny) return;
    const int i = (int)(c % S.nx), j = (int)(c / S.nx);
    const size_t g = gsidx(S.pitch, i, j);
    const int64_t vt = 2 * (int64_t)i + 1 + (int64_t)S.nx * (3 * (int64_t)j + 1);
    const int64_t vu = (int64_t)i + 3 * (int64_t)j * S.nx;
    const int64_t vq = 2 * (int64_t)i + (int64_t)S.nx * (3 * (int64_t)j + 1);
    if (dir == 0) {
        h[vt] = S.f[F_EZ][parity][g];
        h[vu] = S.f[F_HX][parity][g];
        h[vq] = S.f[F_HY][parity][g];
    } else {
        S.f[F_EZ][parity][g] = h[vt];
        S.f[F_HX][parity][g] = h[vu];
        S.f[F_HY][parity][g] = h[vq];
    }
}

__global__ void k_psi_nodes(const TmzDev* __restrict__ sc, int scene, int parity, const int* __restrict__ psi,
                            int n_psi, int64_t base, float* h, int dir) {
    const TmzDev& S = sc[scene];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_psi) return;
    const int p = psi[k];
    const int type = p >> 29, cell = p & ((1 << 29) - 1);
    const int slot = type == 0 ? F_PHXY : (type == 1 ? F_PHYX : (type == 2 ? F_PEZX : F_PEZY));
    const size_t g = gsidx(S.pitch, cell % S.nx, cell / S.nx);
    if (dir == 0) h[base + k] = S.f[slot][parity][g];
    else S.f[slot][parity][g] = h[base + k];
}

// split-field scenes: Ezx = Ez - Ezy where the layer keeps Ezy, Ez elsewhere
__global__ void k_cells_nodes_split(const TmzDev* __restrict__ sc, int scene, int parity, float* h, int dir) {
    const TmzDev& S = sc[scene];
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (int64_t)S.nx * S.ny) return;
    const int i = (int)(c % S.nx), j = (int)(c / S.nx);
    const size_t g = gsidx(S.pitch, i, j);
    const int np = S.split;
    const bool layer = i < np || i > S.nx - np || j < np || j > S.ny - np;
    const int64_t vu = (int64_t)i + 4 * (int64_t)j * S.nx;
    const int64_t vq = 3 * (int64_t)i + (int64_t)S.nx * (4 * (int64_t)j + 1);
    if (dir == 0) {
        const float ezy = layer ? S.f[F_PEZY][parity][g] : 0.f;
        h[vu] = S.f[F_HX][parity][g];
        h[vq] = S.f[F_HY][parity][g];
        h[vq + 1] = S.f[F_EZ][parity][g] - ezy;
        h[vq + 2] = ezy;
    } else {
        S.f[F_HX][parity][g] = h[vu];
        S.f[F_HY][parity][g] = h[vq];
        S.f[F_EZ][parity][g] = h[vq + 1] + h[vq + 2];
        S.f[F_PEZY][parity][g] = h[vq + 2];
    }
}

__global__ void k_graph_src_rec_split(const TmzDev* __restrict__ sc, int scene, const Sample2* __restrict__ samps,
                                      const int* __restrict__ samp_off, float* h, long long n) {
    const TmzDev& S = sc[scene];
    auto q_of = [&](int i, int j) { return 3 * (int64_t)i + (int64_t)S.nx * (4 * (int64_t)j + 1); };
    if (S.src_i >= 0 && n < S.src_len)
        for (int j = S.src_j + (int)threadIdx.x; j < S.src_j1; j += blockDim.x) h[q_of(S.src_i, j) + 1] += S.src_wave[n];
    __syncthreads();
    for (int q = samp_off[scene] + threadIdx.x; q < samp_off[scene + 1]; q += blockDim.x) {
        const Sample2 sp = samps[q];
        float v;
        if (sp.comp == F_EZ) v = h[q_of(sp.i, sp.j) + 1] + h[q_of(sp.i, sp.j) + 2];
        else if (sp.comp == F_HX) v = h[(int64_t)sp.i + 4 * (int64_t)sp.j * S.nx];
        else v = h[q_of(sp.i, sp.j)];
        S.rec[n * S.n_rec + sp.slot] = v;
    }
}

__global__ void k_graph_src_rec(const TmzDev* __restrict__ sc, int scene, const Sample2* __restrict__ samps,
                                const int* __restrict__ samp_off, float* h, long long n) {
    const TmzDev& S = sc[scene];
    if (S.src_i >= 0 && n < S.src_len)
        for (int j = S.src_j + (int)threadIdx.x; j < S.src_j1; j += blockDim.x)
            h[2 * (int64_t)S.src_i + 1 + (int64_t)S.nx * (3 * (int64_t)j + 1)] += S.src_wave[n];
    __syncthreads();
    for (int q = samp_off[scene] + threadIdx.x; q < samp_off[scene + 1]; q += blockDim.x) {
        const Sample2 sp = samps[q];
        int64_t v;
        if (sp.comp == F_EZ) v = 2 * (int64_t)sp.i + 1 + (int64_t)S.nx * (3 * (int64_t)sp.j + 1);
        else if (sp.comp == F_HX) v = (int64_t)sp.i + 3 * (int64_t)sp.j * S.nx;
        else v = 2 * (int64_t)sp.i + (int64_t)S.nx * (3 * (int64_t)sp.j + 1);
        S.rec[n * S.n_rec + sp.slot] = h[v];
    }
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
void graph_free(fdtd_ctx* c) {
    Graph* G = (Graph*)c->graph;
    if (!G) return;
    for (SceneGraph& g : G->g) {
        for (int l = 0; l < 2; l++) {
            cudaFree(g.d_rowptr[l]);
            cudaFree(g.d_col[l]);
            cudaFree(g.d_w[l]);
            cudaFree(g.d_h[l]);
        }
        cudaFree(g.d_psi);
    }
    delete G;
    c->graph = nullptr;
}

static int upload_graph(fdtd_ctx* c, int scene, SceneGraph& g) {
    const Scene2* s = c->s2[scene];
    HostScene h;
    int rc = fetch(c, s, h);
    if (rc) return rc;
    std::vector<int> psi;
    std::vector<int64_t> idx4;
    g.split = h.split;
    if (!h.split) psi_lists(h, psi, idx4);
    g.n_nodes = (h.split ? 4 : 3) * (int64_t)h.nx * h.ny + (int64_t)psi.size();
    g.n_psi = (int)psi.size();
    g.psi_base = 3 * (int64_t)h.nx * h.ny;
    if (g.n_nodes >= ((int64_t)1 << 31)) {
        c->err = "graph: too many nodes for 32-bit indices";
        return FDTD_EINVAL;
    }
    for (int l = 0; l < 2; l++) {
        g.d_rowptr[l] = nullptr; g.d_col[l] = nullptr; g.d_w[l] = nullptr; g.d_h[l] = nullptr;
    }
    g.d_psi = nullptr;
    for (int l = 0; l < 2; l++) {
        std::vector<int> rowptr, col;
        std::vector<float> w;
        if (h.split) {
            build_layer_split(h, l + 1, rowptr, col, w);
        } else {
            build_layer(h, l + 1, psi, idx4, rowptr, col, w);
            if (l == 1) apply_design(h, s, rowptr, col, w, idx4);
        }
        g.nnz[l] = (int64_t)col.size();
        if (cudaMalloc(&g.d_rowptr[l], rowptr.size() * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&g.d_col[l], col.size() * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&g.d_w[l], w.size() * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&g.d_h[l], g.n_nodes * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            c->err = "graph: out of device memory";
            return FDTD_ENOMEM;
        }
        cudaMemcpyAsync(g.d_rowptr[l], rowptr.data(), rowptr.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream);
        cudaMemcpyAsync(g.d_col[l], col.data(), col.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream);
        cudaMemcpyAsync(g.d_w[l], w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream);
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            c->err = std::string("graph upload: ") + cudaGetErrorString(e);
            return FDTD_ECUDA;
        }
    }
    if (cudaMalloc(&g.d_psi, std::max<size_t>(1, psi.size()) * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        c->err = "graph: out of device memory";
        return FDTD_ENOMEM;
    }
    if (!psi.empty()) cudaMemcpyAsync(g.d_psi, psi.data(), psi.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("graph upload: ") + cudaGetErrorString(e);
        return FDTD_ECUDA;
    }
    return FDTD_OK;
}

int graph_prepare(fdtd_ctx* c) {
    if (c->graph) return FDTD_OK;
    Graph* G = new Graph();
    G->g.resize(c->s2.size());
    c->graph = G;
    for (size_t k = 0; k < c->s2.size(); k++) {
        int rc = upload_graph(c, (int)k, G->g[k]);
        if (rc) {
            graph_free(c);
            return rc;
        }
    }
    return FDTD_OK;
}

}  // namespace gem

using namespace gem;

// provided by api.cu
namespace gem {
int step_prepare(fdtd_ctx* c, int64_t n_steps);
}

extern "C" {

int fdtd_step_edgelist(fdtd_ctx* c, int64_t n_steps) {
    NvtxRange nvtx("fdtd_step_edgelist");
    if (!c) return FDTD_EINVAL;
    if (c->dims != 2 || c->s2.empty()) {
        c->err = "the edge-list path is 2D only";
        return FDTD_EINVAL;
    }
    if (ctx_has_slab(c)) {
        c->err = "slab sub-domains step with the implicit-stencil kernels only";
        return FDTD_EINVAL;
    }
    if (n_steps < 0) {
        c->err = "n_steps < 0";
        return FDTD_EINVAL;
    }
    if (n_steps == 0) return FDTD_OK;
    int rc = step_prepare(c, n_steps);
    if (rc) return rc;
    // the graph's weights are frozen from the scene's coefficients when first needed
    rc = graph_prepare(c);
    if (rc) return rc;
    Graph* G = (Graph*)c->graph;
    const int tb = 256;
    for (size_t k = 0; k < c->s2.size(); k++) {
        SceneGraph& g = G->g[k];
        const Scene2* s = c->s2[k];
        const int64_t ncell = (int64_t)s->nx * s->ny;
        if (g.split)
            k_cells_nodes_split<<<(unsigned)((ncell + tb - 1) / tb), tb, 0, c->stream>>>(c->d_scenes, (int)k, c->parity,
                                                                                       g.d_h[0], 0);
        else
            k_cells_nodes<<<(unsigned)((ncell + tb - 1) / tb), tb, 0, c->stream>>>(c->d_scenes, (int)k, c->parity, g.d_h[0], 0);
        if (g.n_psi)
            k_psi_nodes<<<(g.n_psi + tb - 1) / tb, tb, 0, c->stream>>>(c->d_scenes, (int)k, c->parity, g.d_psi, g.n_psi,
                                                                      g.psi_base, g.d_h[0], 0);
        c->launches += g.n_psi ? 2 : 1;
    }
    for (int64_t q = 0; q < n_steps; q++) {
        const long long n = c->t + q;
        for (size_t k = 0; k < c->s2.size(); k++) {
            SceneGraph& g = G->g[k];
            const unsigned blocks = (unsigned)((g.n_nodes + tb - 1) / tb);
            k_mp_layer<<<blocks, tb, 0, c->stream>>>(g.d_rowptr[0], g.d_col[0], g.d_w[0], g.d_h[0], g.d_h[1], g.n_nodes);
            k_mp_layer<<<blocks, tb, 0, c->stream>>>(g.d_rowptr[1], g.d_col[1], g.d_w[1], g.d_h[1], g.d_h[0], g.n_nodes);
            if (g.split)
                k_graph_src_rec_split<<<1, 128, 0, c->stream>>>(c->d_scenes, (int)k, c->d_samp_scene, c->d_samp_off,
                                                                g.d_h[0], n);
            else
                k_graph_src_rec<<<1, 128, 0, c->stream>>>(c->d_scenes, (int)k, c->d_samp_scene, c->d_samp_off, g.d_h[0], n);
            c->launches += 3;
        }
        for (const DftMon& m : c->mons) {
            if (m.plane_k >= 0) continue;
            rc = dft_cells_launch(c, m, n, 1);
            if (rc) return rc;
        }
    }
    for (size_t k = 0; k < c->s2.size(); k++) {
        SceneGraph& g = G->g[k];
        const Scene2* s = c->s2[k];
        const int64_t ncell = (int64_t)s->nx * s->ny;
        if (g.split)
            k_cells_nodes_split<<<(unsigned)((ncell + tb - 1) / tb), tb, 0, c->stream>>>(c->d_scenes, (int)k, c->parity,
                                                                                       g.d_h[0], 1);
        else
            k_cells_nodes<<<(unsigned)((ncell + tb - 1) / tb), tb, 0, c->stream>>>(c->d_scenes, (int)k, c->parity, g.d_h[0], 1);
        if (g.n_psi)
            k_psi_nodes<<<(g.n_psi + tb - 1) / tb, tb, 0, c->stream>>>(c->d_scenes, (int)k, c->parity, g.d_psi, g.n_psi,
                                                                      g.psi_base, g.d_h[0], 1);
        c->launches += g.n_psi ? 2 : 1;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string("edge-list step: ") + cudaGetErrorString(e);
        return FDTD_ECUDA;
    }
    c->t += n_steps;
    return FDTD_OK;
}

int fdtd_export_graph(fdtd_ctx* c, int layer, int64_t* n_nodes, int64_t* n_edges, int32_t* src, int32_t* dst,
                      float* w) {
    if (!c || !n_nodes || !n_edges) return FDTD_EINVAL;
    if (c->dims != 2 || c->s2.empty()) {
        c->err = "graph export is 2D only";
        return FDTD_EINVAL;
    }
    if (ctx_has_slab(c)) {
        c->err = "graph export covers whole grids, not slab sub-domains";
        return FDTD_EINVAL;
    }
    if (layer != 1 && layer != 2) {
        c->err = "layer must be 1 or 2";
        return FDTD_EINVAL;
    }
    const Scene2* s = c->s2[c->cur];
    HostScene h;
    int rc = fetch(c, s, h);
    if (rc) return rc;
    std::vector<int> rowptr, col;
    std::vector<float> ww;
    if (h.split) {
        build_layer_split(h, layer, rowptr, col, ww);
    } else {
        std::vector<int> psi;
        std::vector<int64_t> idx4;
        psi_lists(h, psi, idx4);
        build_layer(h, layer, psi, idx4, rowptr, col, ww);
        if (layer == 2) apply_design(h, s, rowptr, col, ww, idx4);
    }
    const int64_t nn = (int64_t)rowptr.size() - 1;
    *n_nodes = nn;
    *n_edges = (int64_t)col.size();
    if (src && dst && w) {
        for (int64_t v = 0; v < nn; v++)
            for (int e = rowptr[v]; e < rowptr[v + 1]; e++) {
                src[e] = col[e];
                dst[e] = (int32_t)v;
                w[e] = ww[e];
            }
    }
    return FDTD_OK;
}

}  // extern "C"

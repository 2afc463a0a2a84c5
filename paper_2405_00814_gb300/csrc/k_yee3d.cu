// 3D Yee path: the six-component extension of the leapfrog step that the paper
// says follows directly from the 2D scheme (Sec. III-B; Sec. IV-A), with the same
// two layers (H from curl E, then E from curl H), per-cell Ca and Cb from eq. (7)
// for all three E components of a cell, and a CPML of twelve auxiliaries.
//
// Layout: every array is [nz + 2][ny + 2][pitch] FP32 with one zero pad row and
// plane on each side and a 32-cell left pad; cell (i, j, k) sits at
// ((k + 1)(ny + 2) + j + 1) pitch + i + 32, the pitch a multiple of 32 wide
// enough for every kernel's last tile.  Tangential E on the walls i|j|k = 0 is
// never updated (stays zero); the pads are the ghost walls at N.  Three step
// paths: the two-step z-marching kernel (default: two steps per HBM pass), the
// one-step z-marching kernel, and an unfused H launch plus E launch per step
// updating in place.  The z-marching kernels read one copy of every array and
// write the other.  After each step a small launch adds the source and records
// the probes, and the plane DFT accumulates.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "gem_internal.h"

using namespace gem;

// x offset of cell i = 0 in a row: a 32-float (128-byte) left pad puts every
// 128-cell tile row of the fused kernel on a 128-byte line, so a warp's float4
// loads and stores of its row cover whole 32-byte sectors (a partly written
// sector costs the DRAM a read-modify-write), and the staged rows, which start
// 4 cells left of the tile, stay 16-byte aligned
constexpr int PX3 = 32;

enum { G_EX = 0, G_EY, G_EZ, G_HX, G_HY, G_HZ,
       P_EXY, P_EXZ, P_EYZ, P_EYX, P_EZX, P_EZY, P_HXY, P_HXZ, P_HYZ, P_HYX, P_HZX, P_HZY, G_COUNT };

struct Sample3 {
    int i, j, k, comp, slot;
};

struct Scene3 {
    int nx, ny, nz, pitch, rows, planes, npml;
    double dx, dy, dz, dt;
    float* f[G_COUNT];     // current state (the fused kernel writes g and swaps)
    float* g[G_COUNT];
    uint8_t* d_mat;
    float4* d_coef;        // (Ca, Cb/dx, Cb/dy, Cb/dz)
    float* d_prof;         // x: bE cE bH cH [pitch]; y: [rows] x4; z: [planes] x4
    int src_kind, src_i, src_j, src_k, src_comp;
    double src_param;
    std::vector<float> src_samples;
    float* d_src;
    long long src_cap;
    std::vector<Sample3> samples;
    Sample3* d_samp;
    float* d_rec;
    long long rec_cap;
    bool samp_dirty;
    int kernel;            // 0 fused z-marching (default), 1 one H and one E launch per step
    // the two-step kernel's tiling (built for s2_seg): samples by owning tile,
    // and the tiles without CPML reach (d_s2tiles[0, n_int)) and with it (the rest)
    int* d_s2off;
    int* d_s2idx;
    int* d_s2tiles;
    int* d_s2zb;           // z-segment bounds
    int n_s2int, n_s2pml;
    int s2_xs;             // x-slab lanes per warp of the widest tile (the CPML build's slots)
    int s2_seg;
    cudaStream_t aux;      // second stream: the tiles without CPML run beside the others
    cudaEvent_t ev_fork, ev_join;
};

namespace {

const double kC0 = 299792458.0;
const double kMu0 = 4.0e-7 * M_PI;
const double kEps0 = 1.0 / (kMu0 * kC0 * kC0);
const double kPmlM = 3.0;
const double kPmlAlphaMax = 0.05;

struct Dev3 {
    float* f[G_COUNT];
    const uint8_t* mat;
    const float4* coef;
    const float* prof;
    int nx, ny, nz, pitch, rows, planes;
    float cdx, cdy, cdz;    // dt / (mu0 d)
    int has_pml;
};

int fail3(fdtd_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CK3(call, what)                                                                  \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) return fail3(c, FDTD_ECUDA, "%s: %s", what, cudaGetErrorString(e_)); \
    } while (0)

void cpml_pt(double rho, int npml, double delta, double dt, double* b, double* cc) {
    if (rho <= 0.0 || npml <= 0) {
        *b = 0.0;
        *cc = 0.0;
        return;
    }
    const double eta0 = sqrt(kMu0 / kEps0);
    const double smax = 0.8 * (kPmlM + 1.0) / (eta0 * delta);
    const double x = rho / npml;
    const double sig = smax * pow(x, kPmlM);
    const double alp = kPmlAlphaMax * (1.0 - x);
    const double bb = exp(-(sig + alp) * dt / kEps0);
    *b = bb;
    *cc = sig * (bb - 1.0) / (sig + alp);
}

void axis_prof(int n, int npml, double delta, double dt, int len, int off, float* out) {
    // out: bE[len] cE[len] bH[len] cH[len], cell i at i + off
    for (int q = 0; q < 4 * len; q++) out[q] = 0.f;
    if (npml <= 0) return;
    for (int i = 0; i < n; i++) {
        const double xe = i, xh = i + 0.5, lo = npml, hi = n - npml;
        double rE = 0, rH = 0;
        if (xe < lo) rE = lo - xe;
        if (xe > hi) rE = xe - hi;
        if (xh < lo) rH = lo - xh;
        if (xh > hi) rH = xh - hi;
        double b, cc;
        cpml_pt(rE, npml, delta, dt, &b, &cc);
        out[i + off] = (float)b;
        out[len + i + off] = (float)cc;
        cpml_pt(rH, npml, delta, dt, &b, &cc);
        out[2 * len + i + off] = (float)b;
        out[3 * len + i + off] = (float)cc;
    }
}

double wave3(int kind, double p, double t) {
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

Dev3 dev_of(const Scene3* s) {
    Dev3 d;
    for (int q = 0; q < G_COUNT; q++) d.f[q] = s->f[q];
    d.mat = s->d_mat;
    d.coef = s->d_coef;
    d.prof = s->d_prof;
    d.nx = s->nx; d.ny = s->ny; d.nz = s->nz; d.pitch = s->pitch; d.rows = s->rows; d.planes = s->planes;
    d.cdx = (float)(s->dt / (kMu0 * s->dx));
    d.cdy = (float)(s->dt / (kMu0 * s->dy));
    d.cdz = (float)(s->dt / (kMu0 * s->dz));
    d.has_pml = s->npml;
    return d;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
struct P3 {
    const float* p;
    int pitch, rows, planes;
    __device__ float bEx(int i) const { return p[i]; }
    __device__ float cEx(int i) const { return p[pitch + i]; }
    __device__ float bHx(int i) const { return p[2 * pitch + i]; }
    __device__ float cHx(int i) const { return p[3 * pitch + i]; }
    __device__ float bEy(int j) const { return p[4 * pitch + j]; }
    __device__ float cEy(int j) const { return p[4 * pitch + rows + j]; }
    __device__ float bHy(int j) const { return p[4 * pitch + 2 * rows + j]; }
    __device__ float cHy(int j) const { return p[4 * pitch + 3 * rows + j]; }
    __device__ float bEz(int k) const { return p[4 * pitch + 4 * rows + k]; }
    __device__ float cEz(int k) const { return p[4 * pitch + 4 * rows + planes + k]; }
    __device__ float bHz(int k) const { return p[4 * pitch + 4 * rows + 2 * planes + k]; }
    __device__ float cHz(int k) const { return p[4 * pitch + 4 * rows + 3 * planes + k]; }
};

// psi <- b psi + c d; returns d + psi (only where the profile is non-zero)
__device__ __forceinline__ float cpml(float* p, size_t c, float b, float cc, float d) {
    if (b == 0.f && cc == 0.f) return d;
    const float v = b * p[c] + cc * d;
    p[c] = v;
    return d + v;
}

// layer 1: H from curl E (forward differences; the +1 pads are the ghost walls)
__global__ void k_h3(Dev3 S) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= S.nx || j >= S.ny) return;
    const size_t sy = S.pitch, sz = (size_t)S.pitch * S.rows;
    const size_t c = ((size_t)(k + 1) * S.rows + (j + 1)) * S.pitch + (i + PX3);
    const float* ex = S.f[G_EX];
    const float* ey = S.f[G_EY];
    const float* ez = S.f[G_EZ];
    const float exc = ex[c], eyc = ey[c], ezc = ez[c];
    float dezy = ez[c + sy] - ezc, deyz = ey[c + sz] - eyc;
    float dexz = ex[c + sz] - exc, dezx = ez[c + 1] - ezc;
    float deyx = ey[c + 1] - eyc, dexy = ex[c + sy] - exc;
    if (S.has_pml) {
        const P3 pr{S.prof, S.pitch, S.rows, S.planes};
        const float bx = pr.bHx(i + PX3), cx = pr.cHx(i + PX3);
        const float by = pr.bHy(j + 1), cy = pr.cHy(j + 1);
        const float bz = pr.bHz(k + 1), cz = pr.cHz(k + 1);
        dezy = cpml(S.f[P_HXY], c, by, cy, dezy);
        deyz = cpml(S.f[P_HXZ], c, bz, cz, deyz);
        dexz = cpml(S.f[P_HYZ], c, bz, cz, dexz);
        dezx = cpml(S.f[P_HYX], c, bx, cx, dezx);
        deyx = cpml(S.f[P_HZX], c, bx, cx, deyx);
        dexy = cpml(S.f[P_HZY], c, by, cy, dexy);
    }
    S.f[G_HX][c] -= S.cdy * dezy - S.cdz * deyz;
    S.f[G_HY][c] -= S.cdz * dexz - S.cdx * dezx;
    S.f[G_HZ][c] -= S.cdx * deyx - S.cdy * dexy;
}

// layer 2: E from curl H (backward differences); wall components stay zero
__global__ void k_e3(Dev3 S) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= S.nx || j >= S.ny) return;
    const size_t sy = S.pitch, sz = (size_t)S.pitch * S.rows;
    const size_t c = ((size_t)(k + 1) * S.rows + (j + 1)) * S.pitch + (i + PX3);
    const float* hx = S.f[G_HX];
    const float* hy = S.f[G_HY];
    const float* hz = S.f[G_HZ];
    const float4 co = S.coef[S.mat[c]];
    const float hxc = hx[c], hyc = hy[c], hzc = hz[c];
    float dhzy = hzc - hz[c - sy], dhyz = hyc - hy[c - sz];
    float dhxz = hxc - hx[c - sz], dhzx = hzc - hz[c - 1];
    float dhyx = hyc - hy[c - 1], dhxy = hxc - hx[c - sy];
    const bool pml = S.has_pml != 0;
    const P3 pr{S.prof, S.pitch, S.rows, S.planes};
    if (j >= 1 && k >= 1) {
        if (pml) {
            dhzy = cpml(S.f[P_EXY], c, pr.bEy(j + 1), pr.cEy(j + 1), dhzy);
            dhyz = cpml(S.f[P_EXZ], c, pr.bEz(k + 1), pr.cEz(k + 1), dhyz);
        }
        S.f[G_EX][c] = co.x * S.f[G_EX][c] + co.z * dhzy - co.w * dhyz;
    }
    if (i >= 1 && k >= 1) {
        if (pml) {
            dhxz = cpml(S.f[P_EYZ], c, pr.bEz(k + 1), pr.cEz(k + 1), dhxz);
            dhzx = cpml(S.f[P_EYX], c, pr.bEx(i + PX3), pr.cEx(i + PX3), dhzx);
        }
        S.f[G_EY][c] = co.x * S.f[G_EY][c] + co.w * dhxz - co.y * dhzx;
    }
    if (i >= 1 && j >= 1) {
        if (pml) {
            dhyx = cpml(S.f[P_EZX], c, pr.bEx(i + PX3), pr.cEx(i + PX3), dhyx);
            dhxy = cpml(S.f[P_EZY], c, pr.bEy(j + 1), pr.cEy(j + 1), dhxy);
        }
        S.f[G_EZ][c] = co.x * S.f[G_EZ][c] + co.y * dhyx - co.z * dhxy;
    }
}

// ---------------------------------------------------------------------------
// fused z-marching step.  One CTA owns a tile of TXC = 128 cells in x by TYR
// rows in y and a z-segment [kA, kB).  Warp w handles row j = j0 - 1 + w (warp 0
// is the halo row j0 - 1, whose H the owned rows need), each lane 4 consecutive
// cells as float4.  Per plane k:
//   layer 1: H(k) of the warp's row from E(k) (rows j, j+1; the cell right of
//            the lane), E(k+1) and H_old(k); lane 0 also forms Hy, Hz of the
//            cell left of the tile (x0 - 1), recomputed so no other CTA is waited on;
//   layer 2: E(k) of the owned rows from H(k) of the row (left neighbours by
//            warp shuffle), of the row below (shared memory) and H(k-1) of the
//            lane's own cells (registers).
// E planes are staged by cp.async into a shared-memory ring D3 planes ahead of
// use (136-float rows: cells x0-4 .. x0+131); H_old and the material bytes of
// the next plane are prefetched into registers.  Two CTA barriers per plane.
// Reads buffer `in`, writes buffer `out`.  A segment starting above k = 0 first
// recomputes H(kA-1) (warm-up plane, nothing stored).
// ---------------------------------------------------------------------------
constexpr int TXC = 128;           // cells per tile row (32 lanes x 4)
constexpr int TYR = 7;             // owned rows per tile (8 warps with the halo row)
constexpr int NW3 = TYR + 1;       // warps per CTA
constexpr int D3 = 2;              // E planes staged ahead
constexpr int NE3 = D3 + 2;        // E ring slots: planes k .. k + 1 + D3
constexpr int ER3 = TYR + 2;       // staged E rows: j0 - 1 .. j0 + TYR
constexpr int EW4 = (TXC + 8) / 4; // staged E row, float4s: cells x0 - 4 .. x0 + TXC + 3

struct Bufs3 {
    const float* in[G_COUNT];
    float* out[G_COUNT];
};

__device__ __forceinline__ void cpa16(void* smem, const void* gmem, bool valid) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(valid ? 16 : 0) : "memory");
}

size_t fused3_smem() {
    return (size_t)NE3 * 3 * ER3 * EW4 * sizeof(float4)     // E ring
           + (size_t)NW3 * 2 * TXC * sizeof(float)            // H(k) of each row: Hx, Hz
           + 256 * sizeof(float4)                             // coefficient table
           + 4 * TXC * sizeof(float);                         // CPML x-profiles of the tile: bHx cHx bEx cEx
}

__device__ __forceinline__ float f4c(const float4& v, int q) { return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w)); }
__device__ __forceinline__ void f4s(float4& v, int q, float a) {
    if (q == 0) v.x = a; else if (q == 1) v.y = a; else if (q == 2) v.z = a; else v.w = a;
}

// CPML auxiliary of one cell: psi <- b psi + c d, returns d + psi
__device__ __forceinline__ float psi_upd(const float* in, float* out, size_t c, float b, float cc, float d, bool store) {
    if (b == 0.f && cc == 0.f) return d;
    const float v = b * in[c] + cc * d;
    if (store) out[c] = v;
    return d + v;
}

// the same for a lane's four cells at g (16-byte aligned), with their old psi
// p already loaded: cells whose bit in `upd` is clear keep psi (their field
// component is not updated); `nval` cells lie inside the grid and are stored
__device__ __forceinline__ float4 psi4p(const float4 p, float* out, size_t g, float4 b, float4 c, float4 d, bool store,
                                        int nval, unsigned upd) {
    float4 v;
    v.x = (upd & 1u) ? b.x * p.x + c.x * d.x : p.x;
    v.y = (upd & 2u) ? b.y * p.y + c.y * d.y : p.y;
    v.z = (upd & 4u) ? b.z * p.z + c.z * d.z : p.z;
    v.w = (upd & 8u) ? b.w * p.w + c.w * d.w : p.w;
    if (store) {
        if (nval >= 4) {
            *reinterpret_cast<float4*>(out + g) = v;
        } else {
            for (int q = 0; q < nval; q++) out[g + q] = f4c(v, q);
        }
    }
    return make_float4(d.x + v.x, d.y + v.y, d.z + v.z, d.w + v.w);
}

__device__ __forceinline__ float4 psi4(const float* in, float* out, size_t g, float4 b, float4 c, float4 d, bool store,
                                       int nval, unsigned upd) {
    return psi4p(*reinterpret_cast<const float4*>(in + g), out, g, b, c, d, store, nval, upd);
}

__global__ void __launch_bounds__(NW3 * 32, 2) k_yee3d_fused(Dev3 S, Bufs3 B, int segz) {
    extern __shared__ float4 sm4[];
    float4* Eb = sm4;                                                    // [NE3][3][ER3][EW4]
    float* Ht = reinterpret_cast<float*>(sm4 + NE3 * 3 * ER3 * EW4);     // [NW3][2][TXC]
    float4* coef_s = reinterpret_cast<float4*>(Ht + NW3 * 2 * TXC);      // [256]
    float* Xp = reinterpret_cast<float*>(coef_s + 256);                  // [4][TXC]: bHx cHx bEx cEx
    const float* Ef = reinterpret_cast<const float*>(Eb);

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, tid = threadIdx.x;
    const int x0 = blockIdx.x * TXC, j0 = blockIdx.y * TYR;
    const int kA = blockIdx.z * segz, kB = min(kA + segz, S.nz);
    const int pitch = S.pitch, rows = S.rows;
    const int j = j0 - 1 + w;                  // this warp's row
    const int x = x0 + 4 * lane;               // first of this lane's cells
    const bool own_row = w >= 1 && j < S.ny;
    const P3 pr{S.prof, pitch, rows, S.planes};
    const int npml = S.has_pml;
    const bool pml = npml > 0;
    for (int q = tid; q < 256; q += NW3 * 32) coef_s[q] = S.coef[q];
    if (pml)
        for (int q = tid; q < 4 * TXC; q += NW3 * 32) {
            const int a = q / TXC, xc = x0 + q % TXC;
            const bool in = xc < S.nx;
            Xp[q] = !in ? 0.f : (a == 0 ? pr.bHx(xc + PX3) : a == 1 ? pr.cHx(xc + PX3) : a == 2 ? pr.bEx(xc + PX3) : pr.cEx(xc + PX3));
        }

    // CPML reach (conservative; the profiles decide cell by cell)
    const bool lane_px = pml && (x - 1 < npml + 1 || x + 4 >= S.nx - npml - 1);
    const bool row_py = pml && (j < npml + 1 || j >= S.ny - npml - 1);
    const bool jin = j >= 0 && j < S.ny;
    const float hby = row_py && jin ? pr.bHy(j + 1) : 0.f, hcy = row_py && jin ? pr.cHy(j + 1) : 0.f;
    const float eby = row_py && jin ? pr.bEy(j + 1) : 0.f, ecy = row_py && jin ? pr.cEy(j + 1) : 0.f;
    // lane 0's left-halo cell x0 - 1
    const bool halo_x = lane == 0 && x0 > 0;

    // E(p) rows j0-1 .. j0+TYR into ring slot p % NE3; rows past the padded array
    // and planes past nz read as zeros
    auto issue_e = [&](int p) {
        float4* dst = Eb + (size_t)(p % NE3) * 3 * ER3 * EW4;
        for (int q = tid; q < 3 * ER3 * EW4; q += NW3 * 32) {
            const int comp = q / (ER3 * EW4), r = (q / EW4) % ER3, v = q % EW4;
            const int jj = j0 - 1 + r;
            const bool in = jj <= S.ny && p <= S.nz;
            const size_t g = ((size_t)(p + 1) * rows + (jj + 1)) * pitch + x0 - 4 + PX3 + 4 * v;   // cell x0 - 4 + 4v
            cpa16(dst + q, B.in[G_EX + comp] + (in ? g : 0), in);
        }
    };
    auto eidx = [&](int slot, int comp, int r) { return ((slot * 3 + comp) * ER3 + r) * EW4; };

    // this lane's cells in plane p: storage index of cell x
    auto gidx = [&](int p) { return ((size_t)(p + 1) * rows + (j + 1)) * pitch + x + PX3; };
    const bool hrow_ok = j >= -1 && j <= S.ny;
    float4 hxo, hyo, hzo, hxn, hyn, hzn;   // H_old of plane k (o) and k + 1 (n)
    float hym_o = 0.f, hzm_o = 0.f, hym_n = 0.f, hzm_n = 0.f;   // lane 0: H_old at x0 - 1
    uint32_t mo = 0, mn = 0;               // material bytes of the 4 cells
    auto load_plane = [&](int p, float4& hx, float4& hy, float4& hz, float& hym, float& hzm, uint32_t& m) {
        hx = hy = hz = make_float4(0.f, 0.f, 0.f, 0.f);
        hym = hzm = 0.f;
        m = 0;
        if (!hrow_ok || p >= S.nz) return;
        const size_t g = gidx(p);
        hx = *reinterpret_cast<const float4*>(B.in[G_HX] + g);
        hy = *reinterpret_cast<const float4*>(B.in[G_HY] + g);
        hz = *reinterpret_cast<const float4*>(B.in[G_HZ] + g);
        if (own_row) m = *reinterpret_cast<const uint32_t*>(S.mat + g);
        if (halo_x) {
            hym = B.in[G_HY][g - 1];
            hzm = B.in[G_HZ][g - 1];
        }
    };

    const int kf = kA > 0 ? kA - 1 : 0;
    issue_e(kf);
#pragma unroll
    for (int d = 0; d < D3; d++) {
        issue_e(kf + 1 + d);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    load_plane(kf, hxo, hyo, hzo, hym_o, hzm_o, mo);
    float4 hxp = make_float4(0.f, 0.f, 0.f, 0.f), hyp = hxp;   // H(k-1) of the lane's cells
    // one plane; H_old and material of plane k are in the (o) registers, plane
    // k + 1's are loaded into the (n) ones.  The loop alternates the two sets,
    // so no register copy waits on a load that is still in flight.
    auto step = [&](const int k, const float4& hxo, const float4& hyo, const float4& hzo, const float hym_o,
                    const float hzm_o, const uint32_t mo, float4& hxn, float4& hyn, float4& hzn, float& hym_n,
                    float& hzm_n, uint32_t& mn) {
        asm volatile("cp.async.wait_group %0;\n" ::"n"(D3 - 1) : "memory");
        __syncthreads();
        issue_e(k + 1 + D3);   // into the slot plane k - 1 used
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        load_plane(k + 1, hxn, hyn, hzn, hym_n, hzm_n, mn);
        // x-slab lanes: this plane's four x-axis psi, loaded before the H update so
        // their latency overlaps it
        float4 pyx = make_float4(0.f, 0.f, 0.f, 0.f), pzx = pyx, peyx = pyx, pezx = pyx;
        if (lane_px && jin) {
            const size_t g = gidx(k);
            pyx = *reinterpret_cast<const float4*>(B.in[P_HYX] + g);
            pzx = *reinterpret_cast<const float4*>(B.in[P_HZX] + g);
            if (own_row) {
                peyx = *reinterpret_cast<const float4*>(B.in[P_EYX] + g);
                pezx = *reinterpret_cast<const float4*>(B.in[P_EZX] + g);
            }
        }
        const int sc = k % NE3, sn = (k + 1) % NE3;
        const bool kz = pml && (k < npml + 1 || k >= S.nz - npml - 1);
        const bool any_h = lane_px || row_py || kz;
        const bool store = k >= kA;

        // ---- layer 1: H(k) of row j ----
        const int o = 1 + lane;   // float4 slot of the lane's cells in a staged row
        const float4 ex = Eb[eidx(sc, 0, w) + o], ey = Eb[eidx(sc, 1, w) + o], ez = Eb[eidx(sc, 2, w) + o];
        const float4 ezu = Eb[eidx(sc, 2, w + 1) + o], exu = Eb[eidx(sc, 0, w + 1) + o];
        const float4 eyk = Eb[eidx(sn, 1, w) + o], exk = Eb[eidx(sn, 0, w) + o];
        const float ezr = Ef[eidx(sc, 2, w) * 4 + 8 + 4 * lane], eyr = Ef[eidx(sc, 1, w) * 4 + 8 + 4 * lane];
        float4 dezy = make_float4(ezu.x - ez.x, ezu.y - ez.y, ezu.z - ez.z, ezu.w - ez.w);
        float4 deyz = make_float4(eyk.x - ey.x, eyk.y - ey.y, eyk.z - ey.z, eyk.w - ey.w);
        float4 dexz = make_float4(exk.x - ex.x, exk.y - ex.y, exk.z - ex.z, exk.w - ex.w);
        float4 dezx = make_float4(ez.y - ez.x, ez.z - ez.y, ez.w - ez.z, ezr - ez.w);
        float4 deyx = make_float4(ey.y - ey.x, ey.z - ey.y, ey.w - ey.z, eyr - ey.w);
        float4 dexy = make_float4(exu.x - ex.x, exu.y - ex.y, exu.z - ex.z, exu.w - ex.w);
        const int nval = S.nx - x;   // cells of the lane inside the grid (>= 4: all)
        if (any_h && jin) {
            // psi <- b psi + c dF for the lane's four cells, one group per slab axis
            const size_t g = gidx(k);
            const bool st = store && own_row;
            if (row_py) {
                const float4 b4 = make_float4(hby, hby, hby, hby), c4 = make_float4(hcy, hcy, hcy, hcy);
                dezy = psi4(B.in[P_HXY], B.out[P_HXY], g, b4, c4, dezy, st, nval, 15u);
                dexy = psi4(B.in[P_HZY], B.out[P_HZY], g, b4, c4, dexy, st, nval, 15u);
            }
            if (kz) {
                const float bz = pr.bHz(k + 1), cz = pr.cHz(k + 1);
                const float4 b4 = make_float4(bz, bz, bz, bz), c4 = make_float4(cz, cz, cz, cz);
                deyz = psi4(B.in[P_HXZ], B.out[P_HXZ], g, b4, c4, deyz, st, nval, 15u);
                dexz = psi4(B.in[P_HYZ], B.out[P_HYZ], g, b4, c4, dexz, st, nval, 15u);
            }
            if (lane_px) {
                const float4 b4 = *reinterpret_cast<const float4*>(Xp + 0 * TXC + 4 * lane);
                const float4 c4 = *reinterpret_cast<const float4*>(Xp + 1 * TXC + 4 * lane);
                dezx = psi4p(pyx, B.out[P_HYX], g, b4, c4, dezx, st, nval, 15u);
                deyx = psi4p(pzx, B.out[P_HZX], g, b4, c4, deyx, st, nval, 15u);
            }
        }
        const float cdx = S.cdx, cdy = S.cdy, cdz = S.cdz;
        float4 hx, hy, hz;
        hx.x = hxo.x - (cdy * dezy.x - cdz * deyz.x); hx.y = hxo.y - (cdy * dezy.y - cdz * deyz.y);
        hx.z = hxo.z - (cdy * dezy.z - cdz * deyz.z); hx.w = hxo.w - (cdy * dezy.w - cdz * deyz.w);
        hy.x = hyo.x - (cdz * dexz.x - cdx * dezx.x); hy.y = hyo.y - (cdz * dexz.y - cdx * dezx.y);
        hy.z = hyo.z - (cdz * dexz.z - cdx * dezx.z); hy.w = hyo.w - (cdz * dexz.w - cdx * dezx.w);
        hz.x = hzo.x - (cdx * deyx.x - cdy * dexy.x); hz.y = hzo.y - (cdx * deyx.y - cdy * dexy.y);
        hz.z = hzo.z - (cdx * deyx.z - cdy * dexy.z); hz.w = hzo.w - (cdx * deyx.w - cdy * dexy.w);
        // lane 0: Hy, Hz of the cell left of the tile (x0 - 1)
        float hym = 0.f, hzm = 0.f;
        if (halo_x && jin) {
            const int cl = 3;   // staged column of cell x0 - 1
            const float exm = Ef[eidx(sc, 0, w) * 4 + cl], eym = Ef[eidx(sc, 1, w) * 4 + cl];
            const float ezm = Ef[eidx(sc, 2, w) * 4 + cl];
            float dexz_m = Ef[eidx(sn, 0, w) * 4 + cl] - exm;
            float dezx_m = ez.x - ezm, deyx_m = ey.x - eym;
            float dexy_m = Ef[eidx(sc, 0, w + 1) * 4 + cl] - exm;
            if (pml) {
                const size_t gm = gidx(k) - 1;
                const float bz = kz ? pr.bHz(k + 1) : 0.f, cz = kz ? pr.cHz(k + 1) : 0.f;
                dexz_m = psi_upd(B.in[P_HYZ], nullptr, gm, bz, cz, dexz_m, false);
                const float mbx = pr.bHx(x0 - 1 + PX3), mcx = pr.cHx(x0 - 1 + PX3);
                dezx_m = psi_upd(B.in[P_HYX], nullptr, gm, mbx, mcx, dezx_m, false);
                deyx_m = psi_upd(B.in[P_HZX], nullptr, gm, mbx, mcx, deyx_m, false);
                dexy_m = psi_upd(B.in[P_HZY], nullptr, gm, hby, hcy, dexy_m, false);
            }
            hym = hym_o - (cdz * dexz_m - cdx * dezx_m);
            hzm = hzm_o - (cdx * deyx_m - cdy * dexy_m);
        }
        // the row's Hx, Hz for the row above; the owned rows' H is stored
        *reinterpret_cast<float4*>(Ht + (w * 2 + 0) * TXC + 4 * lane) = hx;
        *reinterpret_cast<float4*>(Ht + (w * 2 + 1) * TXC + 4 * lane) = hz;
        if (store && own_row) {
            const size_t g = gidx(k);
            if (x + 3 < S.nx) {
                *reinterpret_cast<float4*>(B.out[G_HX] + g) = hx;
                *reinterpret_cast<float4*>(B.out[G_HY] + g) = hy;
                *reinterpret_cast<float4*>(B.out[G_HZ] + g) = hz;
            } else {
                for (int q = 0; q < 4 && x + q < S.nx; q++) {
                    B.out[G_HX][g + q] = f4c(hx, q);
                    B.out[G_HY][g + q] = f4c(hy, q);
                    B.out[G_HZ][g + q] = f4c(hz, q);
                }
            }
        }
        __syncthreads();

        // ---- layer 2: E(k) of the owned rows ----
        const float hyl0 = __shfl_up_sync(0xffffffffu, hy.w, 1), hzl0 = __shfl_up_sync(0xffffffffu, hz.w, 1);
        if (w >= 1) {
            const float hyl = lane == 0 ? hym : hyl0, hzl = lane == 0 ? hzm : hzl0;
            const float4 hxd = *reinterpret_cast<const float4*>(Ht + ((w - 1) * 2 + 0) * TXC + 4 * lane);
            const float4 hzd = *reinterpret_cast<const float4*>(Ht + ((w - 1) * 2 + 1) * TXC + 4 * lane);
            float4 dhzy = make_float4(hz.x - hzd.x, hz.y - hzd.y, hz.z - hzd.z, hz.w - hzd.w);
            float4 dhyz = make_float4(hy.x - hyp.x, hy.y - hyp.y, hy.z - hyp.z, hy.w - hyp.w);
            float4 dhxz = make_float4(hx.x - hxp.x, hx.y - hxp.y, hx.z - hxp.z, hx.w - hxp.w);
            float4 dhzx = make_float4(hz.x - hzl, hz.y - hz.x, hz.z - hz.y, hz.w - hz.z);
            float4 dhyx = make_float4(hy.x - hyl, hy.y - hy.x, hy.z - hy.y, hy.w - hy.z);
            float4 dhxy = make_float4(hx.x - hxd.x, hx.y - hxd.y, hx.z - hxd.z, hx.w - hxd.w);
            const bool wj = j >= 1, wk = k >= 1;   // Ex, Ez need j >= 1; Ex, Ey need k >= 1
            const unsigned wi = x >= 1 ? 15u : 14u;   // Ey, Ez need i >= 1
            const unsigned mex = (wj && wk) ? 15u : 0u, mey = wk ? wi : 0u, mez = wj ? wi : 0u;
            const size_t g = gidx(k);
            if ((lane_px || row_py || kz) && own_row) {
                if (row_py) {
                    const float4 b4 = make_float4(eby, eby, eby, eby), c4 = make_float4(ecy, ecy, ecy, ecy);
                    dhzy = psi4(B.in[P_EXY], B.out[P_EXY], g, b4, c4, dhzy, store, nval, mex);
                    dhxy = psi4(B.in[P_EZY], B.out[P_EZY], g, b4, c4, dhxy, store, nval, mez);
                }
                if (kz) {
                    const float bz = pr.bEz(k + 1), cz = pr.cEz(k + 1);
                    const float4 b4 = make_float4(bz, bz, bz, bz), c4 = make_float4(cz, cz, cz, cz);
                    dhyz = psi4(B.in[P_EXZ], B.out[P_EXZ], g, b4, c4, dhyz, store, nval, mex);
                    dhxz = psi4(B.in[P_EYZ], B.out[P_EYZ], g, b4, c4, dhxz, store, nval, mey);
                }
                if (lane_px) {
                    const float4 b4 = *reinterpret_cast<const float4*>(Xp + 2 * TXC + 4 * lane);
                    const float4 c4 = *reinterpret_cast<const float4*>(Xp + 3 * TXC + 4 * lane);
                    dhzx = psi4p(peyx, B.out[P_EYX], g, b4, c4, dhzx, store, nval, mey);
                    dhyx = psi4p(pezx, B.out[P_EZX], g, b4, c4, dhyx, store, nval, mez);
                }
            }
            float4 nex = ex, ney = ey, nez = ez;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const float4 co = coef_s[(mo >> (8 * q)) & 255u];
                if (mex & (1u << q)) f4s(nex, q, co.x * f4c(ex, q) + co.z * f4c(dhzy, q) - co.w * f4c(dhyz, q));
                if (mey & (1u << q)) f4s(ney, q, co.x * f4c(ey, q) + co.w * f4c(dhxz, q) - co.y * f4c(dhzx, q));
                if (mez & (1u << q)) f4s(nez, q, co.x * f4c(ez, q) + co.y * f4c(dhyx, q) - co.z * f4c(dhxy, q));
            }
            if (store && own_row) {
                if (x + 3 < S.nx) {
                    *reinterpret_cast<float4*>(B.out[G_EX] + g) = nex;
                    *reinterpret_cast<float4*>(B.out[G_EY] + g) = ney;
                    *reinterpret_cast<float4*>(B.out[G_EZ] + g) = nez;
                } else {
                    for (int q = 0; q < 4 && x + q < S.nx; q++) {
                        B.out[G_EX][g + q] = f4c(nex, q);
                        B.out[G_EY][g + q] = f4c(ney, q);
                        B.out[G_EZ][g + q] = f4c(nez, q);
                    }
                }
            }
        }
        hxp = hx;
        hyp = hy;
    };
    for (int k = kf; k < kB; k += 2) {
        step(k, hxo, hyo, hzo, hym_o, hzm_o, mo, hxn, hyn, hzn, hym_n, hzm_n, mn);
        if (k + 1 >= kB) break;
        step(k + 1, hxn, hyn, hzn, hym_n, hzm_n, mn, hxo, hyo, hzo, hym_o, hzm_o, mo);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

__global__ void k_src_rec3(Dev3 S, int si, int sj, int sk, int scomp, const float* wave, long long wlen,
                           const Sample3* samp, int n_samp, float* rec, long long n) {
    if (threadIdx.x == 0 && si >= 0 && n < wlen) {
        const size_t c = ((size_t)(sk + 1) * S.rows + (sj + 1)) * S.pitch + (si + PX3);
        S.f[scomp][c] += wave[n];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < n_samp; q += blockDim.x) {
        const Sample3 sp = samp[q];
        const size_t c = ((size_t)(sp.k + 1) * S.rows + (sp.j + 1)) * S.pitch + (sp.i + PX3);
        rec[n * n_samp + sp.slot] = S.f[sp.comp][c];
    }
}

__device__ __forceinline__ void kahan3(float& s, float& c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// running DFT over a z plane: acc[pc][f][j][i] = (re, im, comp_re, comp_im)
__global__ void k_dft_plane3(Dev3 S, int plane_k, int comp_mask, const double* freq, int n_freq, double dt,
                             float4* acc, long long n) {
    // the step's twiddles dt e^{-i 2 pi f (n+1) dt}: FP64 phase, once per block
    __shared__ float2 tw[16];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if (tid < n_freq && tid < 16) {
        double ph = freq[tid] * dt * (double)(n + 1);
        ph -= floor(ph);
        double sn, cs;
        sincospi(2.0 * ph, &sn, &cs);
        tw[tid] = make_float2((float)cs * (float)dt, -(float)sn * (float)dt);
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= S.nx || j >= S.ny) return;
    const size_t c = ((size_t)(plane_k + 1) * S.rows + (j + 1)) * S.pitch + (i + PX3);
    const size_t plane = (size_t)S.nx * S.ny;
    const size_t cell = (size_t)j * S.nx + i;
    int pc = 0;
    for (int comp = 0; comp < 3; comp++) {
        if (!(comp_mask & (1 << comp))) continue;
        const float e = S.f[comp][c];
        for (int f = 0; f < n_freq; f++) {
            float4 a = acc[((size_t)pc * n_freq + f) * plane + cell];
            kahan3(a.x, a.z, e * tw[f].x);
            kahan3(a.y, a.w, e * tw[f].y);
            acc[((size_t)pc * n_freq + f) * plane + cell] = a;
        }
        pc++;
    }
}

// the running plane DFT of two steps n and n + 1 in one pass over the
// accumulators: E of step n from the two-step kernel's copy e1 of the plane
// ([3][rows][pitch]), E of step n + 1 from the fields
__global__ void k_dft_plane3_pair(Dev3 S, int plane_k, int comp_mask, const double* freq, int n_freq, double dt,
                                  float4* acc, long long n, const float* e1) {
    __shared__ float2 tw[2][16];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if (tid < 2 * 16) {
        const int s = tid >> 4, f = tid & 15;
        if (f < n_freq) {
            double ph = freq[f] * dt * (double)(n + 1 + s);
            ph -= floor(ph);
            double sn, cs;
            sincospi(2.0 * ph, &sn, &cs);
            tw[s][f] = make_float2((float)cs * (float)dt, -(float)sn * (float)dt);
        }
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= S.nx || j >= S.ny) return;
    const size_t c = ((size_t)(plane_k + 1) * S.rows + (j + 1)) * S.pitch + (i + PX3);
    const size_t c1 = (size_t)(j + 1) * S.pitch + (i + PX3), cs = (size_t)S.rows * S.pitch;
    const size_t plane = (size_t)S.nx * S.ny;
    const size_t cell = (size_t)j * S.nx + i;
    int pc = 0;
    for (int comp = 0; comp < 3; comp++) {
        if (!(comp_mask & (1 << comp))) continue;
        const float ea = e1[comp * cs + c1], eb = S.f[comp][c];
        for (int f = 0; f < n_freq; f++) {
            float4 a = acc[((size_t)pc * n_freq + f) * plane + cell];
            kahan3(a.x, a.z, ea * tw[0][f].x);
            kahan3(a.y, a.w, ea * tw[0][f].y);
            kahan3(a.x, a.z, eb * tw[1][f].x);
            kahan3(a.y, a.w, eb * tw[1][f].y);
            acc[((size_t)pc * n_freq + f) * plane + cell] = a;
        }
        pc++;
    }
}

__global__ void k_dft_cells3(const float* rec, int n_rec, int slot0, int n_cells, const double* freq, int n_freq,
                             double dt, float4* acc, long long n) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n_cells * n_freq) return;
    const int cell = id / n_freq, f = id % n_freq;
    float4 a = acc[id];
    const float e = rec[n * n_rec + slot0 + cell];
    double ph = freq[f] * dt * (double)(n + 1);
    ph -= floor(ph);
    double sn, cs;
    sincospi(2.0 * ph, &sn, &cs);
    kahan3(a.x, a.z, e * ((float)cs * (float)dt));
    kahan3(a.y, a.w, -e * ((float)sn * (float)dt));
    acc[id] = a;
}

// ---------------------------------------------------------------------------
// two-step z-marching kernel (FDTD_OPT_TBLOCK = 2): one HBM pass advances the
// state by two leapfrog steps, n -> n + 2.  A CTA owns TX2 = 120 cells in x by
// TY rows in y and a z-segment [kA, kB).  It computes the first step over the
// owned box grown by two cells on every side in x and y (lanes 0 and 31, warps
// 0, 1 and TY + 2 carry the overlap), so the second step needs nothing that
// another CTA computes.  Warp w handles row r = yo - 2 + w, each lane the four
// cells xo - 4 + 4 lane .. + 3 as float4.  Iteration q (planes kA - 2 .. kB):
//   step 1 at plane q:     H1(q) from E0(q), E0(q + 1) (staged by cp.async)
//                          and H0(q); E1(q) from H1(q) of the row and the row
//                          below (shared memory) and H1(q - 1) (registers);
//                          then the step's source and probe cells, and a copy
//                          of each monitored plane for the DFT launch after;
//   step 2 at plane q - 1: H2(q - 1) from E1(q - 1), E1(q) and E1(q - 1) of the
//                          row above (shared memory, by plane parity); E2(q - 1)
//                          from H2(q - 1) of the row and the row below and
//                          H2(q - 2).
// Values outside the grid are forced to zero at both steps (they are the PEC
// ghost walls).  The first step's CPML auxiliaries wait, by plane parity, for
// the second step: an x-slab lane's in shared-memory slots, the y and z ones in
// thread-local memory.  The CTA's tile comes from a list (the tiles clear of the
// CPML run a build without it).  Reads buffer `in`, writes buffer `out`; only
// the owned cells of the second step are stored.
// ---------------------------------------------------------------------------
constexpr int TX2 = 120;           // owned cells per tile row (lanes 1 .. 30)
constexpr int NE2 = 4;             // E ring slots: planes q .. q + 3
constexpr int MAXP2 = 4;           // plane monitors the kernel copies planes for
constexpr int T2_ROWS = 13;        // owned rows per tile (16 warps)

struct Extra2 {
    const float* wave;             // source waveform: step n adds wave[n] (n < wlen)
    long long wlen;
    int si, sj, sk, scomp;         // source cell and component 0..2 (si < 0: none)
    const Sample3* samp;           // probe and monitor cells
    int n_samp;
    const int* s_off;              // per CTA: [s_off[b], s_off[b + 1]) of s_idx
    const int* s_idx;              // samples each CTA owns, by CTA
    float* rec;                    // rec[n * n_samp + slot]
    int n_mon;                     // plane monitors (<= MAXP2)
    int mon_k[MAXP2], mon_mask[MAXP2];
    float* mon_e1[MAXP2];          // the plane's E after the first step, [3][rows][pitch]
    long long n;                   // index of the first of the two steps
};

// xs: x-slab lanes per warp the CPML build keeps auxiliaries for
template <int TY, bool PML>
constexpr size_t t2_smem(int xs) {
    return ((size_t)NE2 * 3 * (TY + 4) * 32      // E ring [NE2][3][TY + 4][32]
            + (size_t)4 * (TY + 3) * 2 * 32      // H1 rows, E1 rows (two parities), H2 rows
            + 256                                // coefficient table
            + 128                                // x-profiles of the 128 columns
            + (PML ? (size_t)12 * (TY + 3) * xs : 0)) * sizeof(float4);   // x-slab psi, per slab lane
}

__device__ __forceinline__ float4 f4sub(const float4 a, const float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
__device__ __forceinline__ float4 f4add(const float4 a, const float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 f4keep(const float4 v, unsigned m) {
    return make_float4((m & 1u) ? v.x : 0.f, (m & 2u) ? v.y : 0.f, (m & 4u) ? v.z : 0.f, (m & 8u) ? v.w : 0.f);
}
__device__ __forceinline__ float4 f4bc(float a) { return make_float4(a, a, a, a); }
// psi <- b psi + c d for the cells whose bit is set in `upd` (the others keep psi)
__device__ __forceinline__ float4 psi_next(const float4 p, const float4 b, const float4 c, const float4 d, unsigned upd) {
    float4 v;
    v.x = (upd & 1u) ? b.x * p.x + c.x * d.x : p.x;
    v.y = (upd & 2u) ? b.y * p.y + c.y * d.y : p.y;
    v.z = (upd & 4u) ? b.z * p.z + c.z * d.z : p.z;
    v.w = (upd & 8u) ? b.w * p.w + c.w * d.w : p.w;
    return v;
}
// stores the cells of v whose bit is set in m (all four: one 16-byte store)
__device__ __forceinline__ void st4m(float* base, size_t g, const float4 v, unsigned m) {
    if (m == 15u) {
        *reinterpret_cast<float4*>(base + g) = v;
    } else if (m) {
        if (m & 1u) base[g] = v.x;
        if (m & 2u) base[g + 1] = v.y;
        if (m & 4u) base[g + 2] = v.z;
        if (m & 8u) base[g + 3] = v.w;
    }
}
__device__ __forceinline__ float4 ld4(const float* base, size_t g) { return *reinterpret_cast<const float4*>(base + g); }

template <int TY, bool PML>
__global__ void __launch_bounds__((TY + 3) * 32, 1) k_yee3d_t2(Dev3 S, Bufs3 B, Extra2 X, const int* zb, const int* tiles,
                                                                  int gx, int gy, int xs) {
    constexpr int NW = TY + 3, ER = TY + 4, NT = NW * 32;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ float4 sm4[];
    float4* ring = sm4;                                      // [NE2][3][ER][32]
    float4* bH1 = ring + NE2 * 3 * ER * 32;                  // [NW][2][32]: Hx, Hz of step 1
    float4* bE1 = bH1 + NW * 2 * 32;                         // [2][NW][2][32]: Ez, Ex of step 1 by plane parity
    float4* bH2 = bE1 + 2 * NW * 2 * 32;                     // [NW][2][32]: Hx, Hz of step 2
    float4* coef_s = bH2 + NW * 2 * 32;                      // [256]
    float* Xp = reinterpret_cast<float*>(coef_s + 256);      // [4][128]: bHx cHx bEx cEx
    // x-slab lanes' CPML auxiliaries (HYX HZX EYX EZX), a slot per slab lane of
    // each warp (xs per warp): the next plane's stored values (cp.async, one
    // plane ahead) and the first step's values by plane parity
    const int PS = NW * xs;                                      // slots per auxiliary
    float4* px0 = reinterpret_cast<float4*>(Xp + 4 * 128);      // [4][PS]
    float4* px1 = px0 + 4 * PS;                                 // [2][4][PS]

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, tid = threadIdx.x;
    // this CTA's tile of the (gx, gy, z-segments) tiling, from the list; segment
    // bz holds planes [zb[bz], zb[bz + 1])
    const int tile = tiles[blockIdx.x];
    const int bx = tile % gx, by = (tile / gx) % gy, bz = tile / (gx * gy);
    const int xo = bx * TX2, yo = by * TY;
    const int kA = zb[bz], kB = zb[bz + 1];
    const int pitch = S.pitch, rows = S.rows, nx = S.nx, ny = S.ny, nz = S.nz;
    const int r = yo - 2 + w;                  // this warp's row
    const int xc = xo - 4 + 4 * lane;          // first of this lane's cells
    const bool jin = r >= 0 && r < ny;
    unsigned xm = 0, xi1 = 0;                  // cells inside the grid; and with i >= 1
#pragma unroll
    for (int c = 0; c < 4; c++) {
        xm |= (xc + c >= 0 && xc + c < nx) ? (1u << c) : 0u;
        xi1 |= (xc + c >= 1 && xc + c < nx) ? (1u << c) : 0u;
    }
    const bool own_row = w >= 2 && w <= TY + 1 && r < ny;
    const unsigned own_x = (lane >= 1 && lane <= 30) ? xm : 0u;
    const int npml = S.has_pml;
    const bool pml = PML && npml > 0;
    const P3 pr{S.prof, pitch, rows, S.planes};
    for (int q = tid; q < 256; q += NT) coef_s[q] = S.coef[q];
    if (pml)
        for (int q = tid; q < 4 * 128; q += NT) {
            const int a = q >> 7, c = xo - 4 + (q & 127);
            const bool in = c >= 0 && c < nx;
            Xp[q] = !in ? 0.f : (a == 0 ? pr.bHx(c + PX3) : a == 1 ? pr.cHx(c + PX3) : a == 2 ? pr.bEx(c + PX3) : pr.cEx(c + PX3));
        }
    const int sb0 = X.s_off ? X.s_off[tile] : 0, sb1 = X.s_off ? X.s_off[tile + 1] : 0;

    // CPML reach (conservative; the profiles decide cell by cell)
    bool lane_px = pml && xm != 0 && (xc - 1 < npml + 1 || xc + 4 >= nx - npml - 1);
    // this lane's slot among the warp's slab lanes (the host sizes xs for the
    // widest tile; a lane past it would only skip its auxiliaries)
    const int sid = w * xs + __popc(__ballot_sync(FULL, lane_px) & ((1u << lane) - 1u));
    lane_px = lane_px && sid < (w + 1) * xs;
    const bool row_py = pml && jin && (r < npml + 1 || r >= ny - npml - 1);
    const float hby = row_py ? pr.bHy(r + 1) : 0.f, hcy = row_py ? pr.cHy(r + 1) : 0.f;
    const float eby = row_py ? pr.bEy(r + 1) : 0.f, ecy = row_py ? pr.cEy(r + 1) : 0.f;

    const int kf = kA - 2;
    auto gidx = [&](int p) { return ((size_t)(p + 1) * rows + (r + 1)) * pitch + xc + PX3; };
    // E0(p), rows yo-2 .. yo+TY+1, columns xo-4 .. xo+123, into ring slot
    // (p - kf) % NE2; rows and planes outside the padded array and columns past
    // the right pad read as zeros
    auto issue = [&](int p) {
        if (p > kB + 1) return;
        float4* dst = ring + (size_t)((p - kf) & (NE2 - 1)) * 3 * ER * 32;
        const bool pin = p >= -1 && p <= nz;
        for (int e = tid; e < 3 * ER * 32; e += NT) {
            const int v = e & 31, cr = e >> 5;
            const int comp = cr / ER, jj = yo - 2 + (cr - comp * ER);
            const bool in = pin && jj >= -1 && jj <= ny && xo - 4 + 4 * v <= nx;
            const float* src = in ? B.in[G_EX + comp] + ((size_t)(p + 1) * rows + (jj + 1)) * pitch + xo - 4 + 4 * v + PX3
                                  : B.in[G_EX];
            cpa16(dst + e, src, in);
        }
    };
    auto load_h = [&](int p, float4& hx, float4& hy, float4& hz, uint32_t& m) {
        hx = hy = hz = make_float4(0.f, 0.f, 0.f, 0.f);
        m = 0;
        if (!jin || p < 0 || p >= nz || p > kB || xm == 0) return;
        const size_t g = gidx(p);
        hx = ld4(B.in[G_HX], g);
        hy = ld4(B.in[G_HY], g);
        hz = ld4(B.in[G_HZ], g);
        m = *reinterpret_cast<const uint32_t*>(S.mat + g);
    };
    auto issue_pxh = [&](int p) {   // HYX, HZX of plane p (x-slab lanes)
        if (!PML || !lane_px || !jin || p < 0 || p >= nz || p > kB) return;
        const size_t g = gidx(p);
        cpa16(px0 + 0 * PS + sid, B.in[P_HYX] + g, true);
        cpa16(px0 + 1 * PS + sid, B.in[P_HZX] + g, true);
    };
    auto issue_pxe = [&](int p) {   // EYX, EZX of plane p (x-slab lanes)
        if (!PML || !lane_px || !jin || p < 0 || p >= nz || p > kB) return;
        const size_t g = gidx(p);
        cpa16(px0 + 2 * PS + sid, B.in[P_EYX] + g, true);
        cpa16(px0 + 3 * PS + sid, B.in[P_EZX] + g, true);
    };

    // cp.async groups, oldest first, as every iteration q leaves them:
    //   CPML build:  E0(q + 2) | x-psi H(q) | x-psi E(q) | E0(q + 3) | x-psi H(q + 1)
    //   otherwise:   E0(q + 2) | E0(q + 3)
    // (the prologue starts the same sequence with E0 planes kf and kf + 1 first)
    issue(kf);
    issue(kf + 1);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    issue(kf + 2);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    if constexpr (PML) {
        issue_pxh(kf);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        issue_pxe(kf);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    issue(kf + 3);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // the state one iteration hands the next: H0 and material of plane q, the
    // material of plane q - 1, H1(q - 1), E1(q - 1) and H2(q - 2)
    struct St2 {
        float4 hx, hy, hz;
        uint32_t m, mp;
        float4 h1x, h1y, h1z, e1x, e1y, e1z, h2x, h2y;
    };
    St2 s0, s1;
    load_h(kf, s0.hx, s0.hy, s0.hz, s0.m);
    s0.mp = 0;
    s0.h1x = s0.h1y = s0.h1z = s0.e1x = s0.e1y = s0.e1z = s0.h2x = s0.h2y = z4;
    float4 pm[PML ? 2 : 1][PML ? 8 : 1];       // step-1 y and z CPML auxiliaries by plane parity
    asm volatile("cp.async.wait_group 2;\n" ::: "memory");
    __syncthreads();
    const float cdx = S.cdx, cdy = S.cdy, cdz = S.cdz;

    auto body = [&](const int q, const St2& A, St2& Bn) {
        load_h(q + 1, Bn.hx, Bn.hy, Bn.hz, Bn.m);
        const float4* Ec = ring + (size_t)((q - kf) & (NE2 - 1)) * 3 * ER * 32;
        const float4* En = ring + (size_t)((q + 1 - kf) & (NE2 - 1)) * 3 * ER * 32;
        const bool kin1 = q >= 0 && q < nz;
        const unsigned dom1 = (jin && kin1) ? xm : 0u;
        const bool kz1 = pml && kin1 && (q < npml + 1 || q >= nz - npml - 1);
        const bool psi1 = pml && dom1 && (lane_px || row_py || kz1);
        float4* pm1 = pm[PML ? (q & 1) : 0];

        float4* px1q = px1 + (size_t)(q & 1) * 4 * PS + sid;
        if constexpr (PML) asm volatile("cp.async.wait_group 2;\n" ::: "memory");   // x-psi H(q)

        // ---- step 1, layer 1: H1(q) of row r ----
        const float4 ex = Ec[(0 * ER + w) * 32 + lane], ey = Ec[(1 * ER + w) * 32 + lane];
        const float4 ez = Ec[(2 * ER + w) * 32 + lane];
        float4 h1x, h1y, h1z;
        {
            const float4 ezu = Ec[(2 * ER + w + 1) * 32 + lane], exu = Ec[(0 * ER + w + 1) * 32 + lane];
            const float4 eyk = En[(1 * ER + w) * 32 + lane], exk = En[(0 * ER + w) * 32 + lane];
            const float ezr = __shfl_down_sync(FULL, ez.x, 1), eyr = __shfl_down_sync(FULL, ey.x, 1);
            float4 dezy = f4sub(ezu, ez), deyz = f4sub(eyk, ey), dexz = f4sub(exk, ex), dexy = f4sub(exu, ex);
            float4 dezx = make_float4(ez.y - ez.x, ez.z - ez.y, ez.w - ez.z, ezr - ez.w);
            float4 deyx = make_float4(ey.y - ey.x, ey.z - ey.y, ey.w - ey.z, eyr - ey.w);
            if (psi1) {
                const size_t g = gidx(q);
                if (row_py) {
                    const float4 b4 = f4bc(hby), c4 = f4bc(hcy);
                    pm1[0] = psi_next(ld4(B.in[P_HXY], g), b4, c4, dezy, 15u);
                    pm1[1] = psi_next(ld4(B.in[P_HZY], g), b4, c4, dexy, 15u);
                    dezy = f4add(dezy, pm1[0]);
                    dexy = f4add(dexy, pm1[1]);
                }
                if (kz1) {
                    const float4 b4 = f4bc(pr.bHz(q + 1)), c4 = f4bc(pr.cHz(q + 1));
                    pm1[2] = psi_next(ld4(B.in[P_HXZ], g), b4, c4, deyz, 15u);
                    pm1[3] = psi_next(ld4(B.in[P_HYZ], g), b4, c4, dexz, 15u);
                    deyz = f4add(deyz, pm1[2]);
                    dexz = f4add(dexz, pm1[3]);
                }
                if (lane_px) {
                    const float4 b4 = *reinterpret_cast<const float4*>(Xp + 0 * 128 + 4 * lane);
                    const float4 c4 = *reinterpret_cast<const float4*>(Xp + 1 * 128 + 4 * lane);
                    const float4 v4 = psi_next(px0[0 * PS + sid], b4, c4, dezx, 15u);
                    const float4 v5 = psi_next(px0[1 * PS + sid], b4, c4, deyx, 15u);
                    px1q[0 * PS] = v4;
                    px1q[1 * PS] = v5;
                    dezx = f4add(dezx, v4);
                    deyx = f4add(deyx, v5);
                }
            }
            h1x = make_float4(A.hx.x - (cdy * dezy.x - cdz * deyz.x), A.hx.y - (cdy * dezy.y - cdz * deyz.y),
                              A.hx.z - (cdy * dezy.z - cdz * deyz.z), A.hx.w - (cdy * dezy.w - cdz * deyz.w));
            h1y = make_float4(A.hy.x - (cdz * dexz.x - cdx * dezx.x), A.hy.y - (cdz * dexz.y - cdx * dezx.y),
                              A.hy.z - (cdz * dexz.z - cdx * dezx.z), A.hy.w - (cdz * dexz.w - cdx * dezx.w));
            h1z = make_float4(A.hz.x - (cdx * deyx.x - cdy * dexy.x), A.hz.y - (cdx * deyx.y - cdy * dexy.y),
                              A.hz.z - (cdx * deyx.z - cdy * dexy.z), A.hz.w - (cdx * deyx.w - cdy * dexy.w));
            h1x = f4keep(h1x, dom1);
            h1y = f4keep(h1y, dom1);
            h1z = f4keep(h1z, dom1);
        }
        bH1[(w * 2 + 0) * 32 + lane] = h1x;
        bH1[(w * 2 + 1) * 32 + lane] = h1z;
        if constexpr (PML) {
            issue_pxh(q + 1);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        }
        __syncthreads();
        if constexpr (PML) asm volatile("cp.async.wait_group 2;\n" ::: "memory");   // x-psi E(q)

        // ---- step 1, layer 2: E1(q) of rows yo-1 .. yo+TY ----
        float4 e1x = ex, e1y = ey, e1z = ez;
        if (w >= 1) {
            const float4 hxd = bH1[((w - 1) * 2 + 0) * 32 + lane], hzd = bH1[((w - 1) * 2 + 1) * 32 + lane];
            const float hyl = __shfl_up_sync(FULL, h1y.w, 1), hzl = __shfl_up_sync(FULL, h1z.w, 1);
            float4 dhzy = f4sub(h1z, hzd), dhyz = f4sub(h1y, A.h1y), dhxz = f4sub(h1x, A.h1x), dhxy = f4sub(h1x, hxd);
            float4 dhzx = make_float4(h1z.x - hzl, h1z.y - h1z.x, h1z.z - h1z.y, h1z.w - h1z.z);
            float4 dhyx = make_float4(h1y.x - hyl, h1y.y - h1y.x, h1y.z - h1y.y, h1y.w - h1y.z);
            // Ex needs j, k >= 1; Ey i, k >= 1; Ez i, j >= 1 (the rest are PEC walls)
            const unsigned mex = (r >= 1 && q >= 1) ? dom1 : 0u, mey = q >= 1 ? (dom1 ? xi1 : 0u) : 0u;
            const unsigned mez = r >= 1 ? (dom1 ? xi1 : 0u) : 0u;
            if (psi1) {
                const size_t g = gidx(q);
                if (row_py) {
                    const float4 b4 = f4bc(eby), c4 = f4bc(ecy);
                    pm1[4] = psi_next(ld4(B.in[P_EXY], g), b4, c4, dhzy, mex);
                    pm1[5] = psi_next(ld4(B.in[P_EZY], g), b4, c4, dhxy, mez);
                    dhzy = f4add(dhzy, pm1[4]);
                    dhxy = f4add(dhxy, pm1[5]);
                }
                if (kz1) {
                    const float4 b4 = f4bc(pr.bEz(q + 1)), c4 = f4bc(pr.cEz(q + 1));
                    pm1[6] = psi_next(ld4(B.in[P_EXZ], g), b4, c4, dhyz, mex);
                    pm1[7] = psi_next(ld4(B.in[P_EYZ], g), b4, c4, dhxz, mey);
                    dhyz = f4add(dhyz, pm1[6]);
                    dhxz = f4add(dhxz, pm1[7]);
                }
                if (lane_px) {
                    const float4 b4 = *reinterpret_cast<const float4*>(Xp + 2 * 128 + 4 * lane);
                    const float4 c4 = *reinterpret_cast<const float4*>(Xp + 3 * 128 + 4 * lane);
                    const float4 va = psi_next(px0[2 * PS + sid], b4, c4, dhzx, mey);
                    const float4 vb = psi_next(px0[3 * PS + sid], b4, c4, dhyx, mez);
                    px1q[2 * PS] = va;
                    px1q[3 * PS] = vb;
                    dhzx = f4add(dhzx, va);
                    dhyx = f4add(dhyx, vb);
                }
            }
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const float4 co = coef_s[(A.m >> (8 * c)) & 255u];
                if (mex & (1u << c)) f4s(e1x, c, co.x * f4c(ex, c) + co.z * f4c(dhzy, c) - co.w * f4c(dhyz, c));
                if (mey & (1u << c)) f4s(e1y, c, co.x * f4c(ey, c) + co.w * f4c(dhxz, c) - co.y * f4c(dhzx, c));
                if (mez & (1u << c)) f4s(e1z, c, co.x * f4c(ez, c) + co.y * f4c(dhyx, c) - co.z * f4c(dhxy, c));
            }
            // the first step's source, in every CTA that computes its cell
            if (X.si >= xc && X.si < xc + 4 && r == X.sj && q == X.sk && X.n < X.wlen) {
                const float s = X.wave[X.n];
                const int c = X.si - xc;
                if (X.scomp == 0) f4s(e1x, c, f4c(e1x, c) + s);
                else if (X.scomp == 1) f4s(e1y, c, f4c(e1y, c) + s);
                else f4s(e1z, c, f4c(e1z, c) + s);
            }
            float4* be = bE1 + (size_t)(((q - kf) & 1) * NW + w) * 2 * 32;
            be[lane] = e1z;
            be[32 + lane] = e1x;
        }
        // the first step's probe and monitor cells this CTA owns
        for (int s = sb0; s < sb1; s++) {
            const Sample3 sp = X.samp[X.s_idx[s]];
            if (sp.k == q && sp.j == r && sp.i >= xc && sp.i < xc + 4) {
                const int c = sp.i - xc;
                const float4 v = sp.comp == G_EX ? e1x : sp.comp == G_EY ? e1y : sp.comp == G_EZ ? e1z
                               : sp.comp == G_HX ? h1x : sp.comp == G_HY ? h1y : h1z;
                X.rec[X.n * X.n_samp + sp.slot] = f4c(v, c);
            }
        }
        // a monitored plane's E after the first step, for the DFT launch that
        // accumulates both steps after this kernel
        if (X.n_mon > 0 && own_row && own_x && q >= kA && q < kB)
            for (int m = 0; m < X.n_mon; m++) {
                if (X.mon_k[m] != q) continue;
                const size_t g = (size_t)(r + 1) * pitch + xc + PX3, cs = (size_t)rows * pitch;
                if (X.mon_mask[m] & 1) st4m(X.mon_e1[m], g, e1x, own_x);
                if (X.mon_mask[m] & 2) st4m(X.mon_e1[m] + cs, g, e1y, own_x);
                if (X.mon_mask[m] & 4) st4m(X.mon_e1[m] + 2 * cs, g, e1z, own_x);
            }

        // ---- step 2, layer 1: H2(q - 1) of rows yo-1 .. yo+TY-1 ----
        const int p2 = q - 1;
        const bool kin2 = p2 >= 0 && p2 < nz;
        const unsigned dom2 = (jin && kin2) ? xm : 0u;
        const bool kz2 = pml && kin2 && (p2 < npml + 1 || p2 >= nz - npml - 1);
        const bool psi2 = pml && dom2 && (lane_px || row_py || kz2);
        const unsigned om = (own_row && p2 >= kA) ? own_x : 0u;   // cells of plane p2 this CTA stores
        const float4* pm2 = pm[PML ? (p2 & 1) : 0];
        const float4* px2 = px1 + (size_t)(p2 & 1) * 4 * PS + sid;   // x-slab psi of step 1 at plane p2
        float4 h2x = z4, h2y = z4, h2z = z4;
        const bool do_h2 = w >= 1 && w <= TY + 1 && q >= kA;
        if (do_h2) {
            const float4* be = bE1 + (size_t)(((p2 - kf) & 1) * NW + w + 1) * 2 * 32;
            const float4 ezu = be[lane], exu = be[32 + lane];
            const float ezr = __shfl_down_sync(FULL, A.e1z.x, 1), eyr = __shfl_down_sync(FULL, A.e1y.x, 1);
            float4 dezy = f4sub(ezu, A.e1z), deyz = f4sub(e1y, A.e1y), dexz = f4sub(e1x, A.e1x), dexy = f4sub(exu, A.e1x);
            float4 dezx = make_float4(A.e1z.y - A.e1z.x, A.e1z.z - A.e1z.y, A.e1z.w - A.e1z.z, ezr - A.e1z.w);
            float4 deyx = make_float4(A.e1y.y - A.e1y.x, A.e1y.z - A.e1y.y, A.e1y.w - A.e1y.z, eyr - A.e1y.w);
            if (psi2) {
                const size_t g = gidx(p2);
                if (row_py) {
                    const float4 b4 = f4bc(hby), c4 = f4bc(hcy);
                    const float4 v0 = psi_next(pm2[0], b4, c4, dezy, 15u), v1 = psi_next(pm2[1], b4, c4, dexy, 15u);
                    st4m(B.out[P_HXY], g, v0, om);
                    st4m(B.out[P_HZY], g, v1, om);
                    dezy = f4add(dezy, v0);
                    dexy = f4add(dexy, v1);
                }
                if (kz2) {
                    const float4 b4 = f4bc(pr.bHz(p2 + 1)), c4 = f4bc(pr.cHz(p2 + 1));
                    const float4 v2 = psi_next(pm2[2], b4, c4, deyz, 15u), v3 = psi_next(pm2[3], b4, c4, dexz, 15u);
                    st4m(B.out[P_HXZ], g, v2, om);
                    st4m(B.out[P_HYZ], g, v3, om);
                    deyz = f4add(deyz, v2);
                    dexz = f4add(dexz, v3);
                }
                if (lane_px) {
                    const float4 b4 = *reinterpret_cast<const float4*>(Xp + 0 * 128 + 4 * lane);
                    const float4 c4 = *reinterpret_cast<const float4*>(Xp + 1 * 128 + 4 * lane);
                    const float4 v4 = psi_next(px2[0 * PS], b4, c4, dezx, 15u), v5 = psi_next(px2[1 * PS], b4, c4, deyx, 15u);
                    st4m(B.out[P_HYX], g, v4, om);
                    st4m(B.out[P_HZX], g, v5, om);
                    dezx = f4add(dezx, v4);
                    deyx = f4add(deyx, v5);
                }
            }
            h2x = make_float4(A.h1x.x - (cdy * dezy.x - cdz * deyz.x), A.h1x.y - (cdy * dezy.y - cdz * deyz.y),
                              A.h1x.z - (cdy * dezy.z - cdz * deyz.z), A.h1x.w - (cdy * dezy.w - cdz * deyz.w));
            h2y = make_float4(A.h1y.x - (cdz * dexz.x - cdx * dezx.x), A.h1y.y - (cdz * dexz.y - cdx * dezx.y),
                              A.h1y.z - (cdz * dexz.z - cdx * dezx.z), A.h1y.w - (cdz * dexz.w - cdx * dezx.w));
            h2z = make_float4(A.h1z.x - (cdx * deyx.x - cdy * dexy.x), A.h1z.y - (cdx * deyx.y - cdy * dexy.y),
                              A.h1z.z - (cdx * deyx.z - cdy * dexy.z), A.h1z.w - (cdx * deyx.w - cdy * dexy.w));
            h2x = f4keep(h2x, dom2);
            h2y = f4keep(h2y, dom2);
            h2z = f4keep(h2z, dom2);
            bH2[(w * 2 + 0) * 32 + lane] = h2x;
            bH2[(w * 2 + 1) * 32 + lane] = h2z;
            if (om) {
                const size_t g = gidx(p2);
                st4m(B.out[G_HX], g, h2x, om);
                st4m(B.out[G_HY], g, h2y, om);
                st4m(B.out[G_HZ], g, h2z, om);
            }
        }
        // planes q + 1 and q + 2 staged (four newer groups, one without the
        // CPML, may still be in flight); then plane q's slot takes plane q + NE2
        if constexpr (PML)
            asm volatile("cp.async.wait_group 4;\n" ::: "memory");
        else
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        __syncthreads();
        if constexpr (PML) {
            issue_pxe(q + 1);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        }
        issue(q + NE2);
        asm volatile("cp.async.commit_group;\n" ::: "memory");

        // ---- step 2, layer 2: E2(q - 1) of the owned rows ----
        if (w >= 2 && w <= TY + 1 && p2 >= kA) {
            const float4 hxd = bH2[((w - 1) * 2 + 0) * 32 + lane], hzd = bH2[((w - 1) * 2 + 1) * 32 + lane];
            const float hyl = __shfl_up_sync(FULL, h2y.w, 1), hzl = __shfl_up_sync(FULL, h2z.w, 1);
            float4 dhzy = f4sub(h2z, hzd), dhyz = f4sub(h2y, A.h2y), dhxz = f4sub(h2x, A.h2x), dhxy = f4sub(h2x, hxd);
            float4 dhzx = make_float4(h2z.x - hzl, h2z.y - h2z.x, h2z.z - h2z.y, h2z.w - h2z.z);
            float4 dhyx = make_float4(h2y.x - hyl, h2y.y - h2y.x, h2y.z - h2y.y, h2y.w - h2y.z);
            const unsigned mex = (r >= 1 && p2 >= 1) ? dom2 : 0u, mey = p2 >= 1 ? (dom2 ? xi1 : 0u) : 0u;
            const unsigned mez = r >= 1 ? (dom2 ? xi1 : 0u) : 0u;
            if (psi2) {
                const size_t g = gidx(p2);
                if (row_py) {
                    const float4 b4 = f4bc(eby), c4 = f4bc(ecy);
                    const float4 v6 = psi_next(pm2[4], b4, c4, dhzy, mex), v7 = psi_next(pm2[5], b4, c4, dhxy, mez);
                    st4m(B.out[P_EXY], g, v6, om);
                    st4m(B.out[P_EZY], g, v7, om);
                    dhzy = f4add(dhzy, v6);
                    dhxy = f4add(dhxy, v7);
                }
                if (kz2) {
                    const float4 b4 = f4bc(pr.bEz(p2 + 1)), c4 = f4bc(pr.cEz(p2 + 1));
                    const float4 v8 = psi_next(pm2[6], b4, c4, dhyz, mex), v9 = psi_next(pm2[7], b4, c4, dhxz, mey);
                    st4m(B.out[P_EXZ], g, v8, om);
                    st4m(B.out[P_EYZ], g, v9, om);
                    dhyz = f4add(dhyz, v8);
                    dhxz = f4add(dhxz, v9);
                }
                if (lane_px) {
                    const float4 b4 = *reinterpret_cast<const float4*>(Xp + 2 * 128 + 4 * lane);
                    const float4 c4 = *reinterpret_cast<const float4*>(Xp + 3 * 128 + 4 * lane);
                    const float4 va = psi_next(px2[2 * PS], b4, c4, dhzx, mey), vb = psi_next(px2[3 * PS], b4, c4, dhyx, mez);
                    st4m(B.out[P_EYX], g, va, om);
                    st4m(B.out[P_EZX], g, vb, om);
                    dhzx = f4add(dhzx, va);
                    dhyx = f4add(dhyx, vb);
                }
            }
            float4 e2x = A.e1x, e2y = A.e1y, e2z = A.e1z;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const float4 co = coef_s[(A.mp >> (8 * c)) & 255u];
                if (mex & (1u << c)) f4s(e2x, c, co.x * f4c(A.e1x, c) + co.z * f4c(dhzy, c) - co.w * f4c(dhyz, c));
                if (mey & (1u << c)) f4s(e2y, c, co.x * f4c(A.e1y, c) + co.w * f4c(dhxz, c) - co.y * f4c(dhzx, c));
                if (mez & (1u << c)) f4s(e2z, c, co.x * f4c(A.e1z, c) + co.y * f4c(dhyx, c) - co.z * f4c(dhxy, c));
            }
            if (om) {
                const size_t g = gidx(p2);
                st4m(B.out[G_EX], g, e2x, om);
                st4m(B.out[G_EY], g, e2y, om);
                st4m(B.out[G_EZ], g, e2z, om);
            }
        }
        Bn.h2x = h2x;
        Bn.h2y = h2y;
        Bn.h1x = h1x; Bn.h1y = h1y; Bn.h1z = h1z;
        Bn.e1x = e1x; Bn.e1y = e1y; Bn.e1z = e1z;
        Bn.mp = A.m;
    };
    for (int q = kf; q <= kB; q++) {
        body(q, s0, s1);
        s0 = s1;
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}


__global__ void k_finite3(Dev3 S, int* bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= S.nx || j >= S.ny) return;
    const size_t c = ((size_t)(k + 1) * S.rows + (j + 1)) * S.pitch + (i + PX3);
    float v = 0.f;
    for (int q = 0; q < 6; q++) v += S.f[q][c];
    if (!isfinite(v)) atomicOr(bad, 1);
}

void scene3_free(Scene3* s) {
    if (!s) return;
    for (int q = 0; q < G_COUNT; q++) {
        if (s->f[q]) cudaFree(s->f[q]);
        if (s->g[q]) cudaFree(s->g[q]);
    }
    if (s->d_mat) cudaFree(s->d_mat);
    if (s->d_coef) cudaFree(s->d_coef);
    if (s->d_prof) cudaFree(s->d_prof);
    if (s->d_src) cudaFree(s->d_src);
    if (s->d_samp) cudaFree(s->d_samp);
    if (s->d_rec) cudaFree(s->d_rec);
    if (s->d_s2off) cudaFree(s->d_s2off);
    if (s->d_s2idx) cudaFree(s->d_s2idx);
    if (s->d_s2tiles) cudaFree(s->d_s2tiles);
    if (s->d_s2zb) cudaFree(s->d_s2zb);
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    if (s->aux) cudaStreamDestroy(s->aux);
    delete s;
}

Scene3* S3(fdtd_ctx* c) { return c->s3; }

int ensure3(fdtd_ctx* c, int64_t t_end) {
    Scene3* s = S3(c);
    if (s->src_kind >= 0 && s->src_cap < t_end) {
        const int64_t cap = std::max<int64_t>(std::max<int64_t>(t_end, 2 * s->src_cap), 1024);
        std::vector<float> w((size_t)cap);
        for (int64_t n = 0; n < cap; n++)
            w[n] = s->src_kind == FDTD_SRC_SAMPLED ? (n < (int64_t)s->src_samples.size() ? s->src_samples[n] : 0.f)
                                                  : (float)wave3(s->src_kind, s->src_param, (double)(n + 1) * s->dt);
        float* d = nullptr;
        if (cudaMalloc(&d, cap * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return fail3(c, FDTD_ENOMEM, "source waveform");
        }
        CK3(cudaMemcpyAsync(d, w.data(), cap * sizeof(float), cudaMemcpyHostToDevice, c->stream), "waveform");
        CK3(cudaStreamSynchronize(c->stream), "waveform");
        if (s->d_src) cudaFree(s->d_src);
        s->d_src = d;
        s->src_cap = cap;
    }
    const int nrec = (int)s->samples.size();
    if (nrec > 0 && s->rec_cap < t_end) {
        const int64_t cap = std::max<int64_t>(std::max<int64_t>(t_end, 2 * s->rec_cap), 1024);
        float* d = nullptr;
        if (cudaMalloc(&d, (size_t)cap * nrec * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return fail3(c, FDTD_ENOMEM, "sample record");
        }
        CK3(cudaMemsetAsync(d, 0, (size_t)cap * nrec * sizeof(float), c->stream), "record");
        if (s->d_rec)
            CK3(cudaMemcpyAsync(d, s->d_rec, (size_t)s->rec_cap * nrec * sizeof(float), cudaMemcpyDeviceToDevice,
                                c->stream), "record");
        CK3(cudaStreamSynchronize(c->stream), "record");
        if (s->d_rec) cudaFree(s->d_rec);
        s->d_rec = d;
        s->rec_cap = cap;
    }
    if (s->samp_dirty) {
        if (s->d_samp) cudaFree(s->d_samp);
        s->d_samp = nullptr;
        if (cudaMalloc(&s->d_samp, std::max<size_t>(1, s->samples.size()) * sizeof(Sample3)) != cudaSuccess) {
            cudaGetLastError();
            return fail3(c, FDTD_ENOMEM, "samples");
        }
        if (!s->samples.empty())
            CK3(cudaMemcpyAsync(s->d_samp, s->samples.data(), s->samples.size() * sizeof(Sample3),
                                cudaMemcpyHostToDevice, c->stream), "samples");
        CK3(cudaStreamSynchronize(c->stream), "samples");
        s->samp_dirty = false;
        s->s2_seg = -1;
    }
    return FDTD_OK;
}

int slot3(int comp) { return (comp >= FDTD_EX && comp <= FDTD_HZ) ? comp : -1; }

}  // namespace

namespace gem {

int fdtd_create3(const fdtd_grid* g, double dx, double dt, double courant, const uint8_t* mat,
                 const fdtd_material* table, int n_mat, void* stream, fdtd_ctx** out) {
    fdtd_ctx* c = new fdtd_ctx();
    c->dims = 3;
    c->stream = (cudaStream_t)stream;
    c->s3 = nullptr;
    c->cur = 0; c->t = 0; c->parity = 0; c->launches = 0;
    c->opt_kernel = 0; c->opt_tblock = 2; c->opt_segment = 0; c->opt_warps = 8; c->opt_segment_b = 0; c->opt_warps_b = 2; c->opt_playout = 0;
    c->dirty = true;
    c->d_scenes = nullptr; c->d_tasks = nullptr; c->d_tasks_b = nullptr; c->n_tasks_b = 0; c->warps_b = 2; c->d_tasks_l = nullptr; c->n_tasks_l = 0; c->warps_l = 4; c->d_tasks_s = nullptr; c->n_tasks_s = 0; c->d_tasks_bd = nullptr; c->n_tasks_bd = 0;
    c->d_dft = nullptr; c->n_dft = 0; c->opt_adj_store = 1;
    c->d_tasks_n = nullptr; c->n_tasks_n = 0; c->task_narrow = -1; c->task_pers = -1;
    c->opt_check_every = 0; c->d_bad = nullptr; c->h_bad = nullptr;
    c->aux = c->aux2 = nullptr; c->ev_fork = c->ev_join = c->ev_join2 = nullptr;
    c->d_samp = nullptr; c->d_samp_scene = nullptr; c->d_samp_off = nullptr;
    c->n_tasks = 0; c->task_tb = c->task_seg = -1; c->graph = nullptr; c->adj = nullptr;
    *out = c;
    if (!mat || !table) return fail3(c, FDTD_EINVAL, "NULL material map or table");
    if (g->nx < 4 || g->ny < 4 || g->nz < 4) return fail3(c, FDTD_EINVAL, "3D grid needs >= 4 cells per axis");
    if (!(dx > 0)) return fail3(c, FDTD_EINVAL, "dx must be > 0");
    const double dy = g->dy > 0 ? g->dy : dx, dz = g->dz > 0 ? g->dz : dx;
    int npml = 0;
    if (g->boundary == FDTD_CPML) {
        npml = g->pml_cells;
        if (npml < 1 || 2 * npml + 2 > std::min(g->nx, std::min(g->ny, g->nz)))
            return fail3(c, FDTD_EINVAL, "pml_cells %d does not fit the grid", npml);
    } else if (g->boundary != FDTD_PEC) {
        return fail3(c, FDTD_EINVAL, "unknown boundary %d", g->boundary);
    }
    const double lim = 1.0 / (kC0 * sqrt(1.0 / (dx * dx) + 1.0 / (dy * dy) + 1.0 / (dz * dz)));
    if (dt <= 0) {
        if (!(courant > 0 && courant <= 1.0)) return fail3(c, FDTD_EINVAL, "courant factor must be in (0, 1]");
        dt = courant * lim;
    } else if (dt > lim) {
        return fail3(c, FDTD_EUNSTABLE, "dt %.6g s exceeds the 3D Courant limit %.6g s", dt, lim);
    }
    if (n_mat < 1 || n_mat > 255) return fail3(c, FDTD_EINVAL, "n_mat %d outside 1..255", n_mat);
    for (int m = 0; m < n_mat; m++) {
        if (!(table[m].eps_r > 0) || table[m].mu_r != 1.0 || !(table[m].sigma >= 0))
            return fail3(c, FDTD_EINVAL, "material %d: need eps_r > 0, mu_r = 1, sigma >= 0", m);
    }
    const int64_t ncell = (int64_t)g->nx * g->ny * g->nz;
    for (int64_t q = 0; q < ncell; q++)
        if (mat[q] >= n_mat) return fail3(c, FDTD_EINVAL, "material index %d >= n_mat %d", mat[q], n_mat);

    Scene3* s = new Scene3();
    for (int q = 0; q < G_COUNT; q++) s->f[q] = s->g[q] = nullptr;
    s->d_mat = nullptr; s->d_coef = nullptr; s->d_prof = nullptr; s->d_src = nullptr; s->d_samp = nullptr;
    s->d_rec = nullptr;
    s->d_s2off = nullptr; s->d_s2idx = nullptr; s->d_s2tiles = nullptr; s->d_s2zb = nullptr;
    s->n_s2int = s->n_s2pml = 0; s->s2_seg = -1;
    s->s2_xs = 1;
    s->aux = nullptr; s->ev_fork = s->ev_join = nullptr;
    s->nx = g->nx; s->ny = g->ny; s->nz = g->nz; s->npml = npml;
    s->dx = dx; s->dy = dy; s->dz = dz; s->dt = dt;
    // room for the unfused kernels' neighbours and the fused kernel's last tile,
    // whose staged rows reach cell x0 + TXC + 3 (storage column x0 + TXC + 3 + PX3)
    // and the two-step kernel's last tile, whose lanes reach cell 120 ntx + 3
    s->pitch = (std::max(std::max(g->nx + PX3 + 40, (g->nx + TXC - 1) / TXC * TXC + PX3 + 8),
                         (g->nx + TX2 - 1) / TX2 * TX2 + PX3 + 8) + 31) / 32 * 32;
    s->rows = g->ny + 2;
    s->planes = g->nz + 2;
    s->src_kind = -1; s->src_i = s->src_j = s->src_k = -1; s->src_comp = G_EZ; s->src_param = 0; s->src_cap = 0;
    s->rec_cap = 0;
    s->samp_dirty = true;
    c->s3 = s;
    const size_t n = (size_t)s->pitch * s->rows * s->planes;
    for (int q = 0; q < G_COUNT; q++) {
        // psi arrays exist only when there is a CPML
        if (q >= P_EXY && npml == 0) break;
        // two copies: the fused kernel reads one and writes the other
        if (cudaMalloc(&s->f[q], n * sizeof(float)) != cudaSuccess || cudaMalloc(&s->g[q], n * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return fail3(c, FDTD_ENOMEM, "3D field array of %zu bytes", n * sizeof(float));
        }
        CK3(cudaMemsetAsync(s->f[q], 0, n * sizeof(float), c->stream), "memset");
        CK3(cudaMemsetAsync(s->g[q], 0, n * sizeof(float), c->stream), "memset");
    }
    std::vector<uint8_t> pm(n, 0);
    for (int k = 0; k < s->nz; k++)
        for (int j = 0; j < s->ny; j++)
            memcpy(&pm[((size_t)(k + 1) * s->rows + j + 1) * s->pitch + PX3], mat + ((size_t)k * s->ny + j) * s->nx, s->nx);
    std::vector<float4> co(256, make_float4(0, 0, 0, 0));
    for (int m = 0; m < n_mat; m++) {
        const double eps = kEps0 * table[m].eps_r;
        const double am = 1.0 - table[m].sigma * dt / (2.0 * eps), ap = 1.0 + table[m].sigma * dt / (2.0 * eps);
        const double cb = dt / (ap * eps);
        co[m] = make_float4((float)(am / ap), (float)(cb / dx), (float)(cb / dy), (float)(cb / dz));
    }
    std::vector<float> prof(4 * ((size_t)s->pitch + s->rows + s->planes), 0.f);
    axis_prof(s->nx, npml, dx, dt, s->pitch, PX3, prof.data());
    axis_prof(s->ny, npml, dy, dt, s->rows, 1, prof.data() + 4 * s->pitch);
    axis_prof(s->nz, npml, dz, dt, s->planes, 1, prof.data() + 4 * s->pitch + 4 * s->rows);
    if (cudaMalloc(&s->d_mat, n) != cudaSuccess || cudaMalloc(&s->d_coef, 256 * sizeof(float4)) != cudaSuccess ||
        cudaMalloc(&s->d_prof, prof.size() * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return fail3(c, FDTD_ENOMEM, "3D material / tables");
    }
    CK3(cudaMemcpyAsync(s->d_mat, pm.data(), n, cudaMemcpyHostToDevice, c->stream), "upload");
    CK3(cudaMemcpyAsync(s->d_coef, co.data(), 256 * sizeof(float4), cudaMemcpyHostToDevice, c->stream), "upload");
    CK3(cudaMemcpyAsync(s->d_prof, prof.data(), prof.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream), "upload");
    CK3(cudaStreamSynchronize(c->stream), "upload");
    return FDTD_OK;
}

void fdtd_destroy3(fdtd_ctx* c) {
    if (c && c->s3) {
        scene3_free(c->s3);
        c->s3 = nullptr;
    }
}

int fdtd_set_source3(fdtd_ctx* c, int kind, int i, int j, int k, int comp, const double* params,
                     const float* samples, int64_t n_samples) {
    Scene3* s = S3(c);
    if (!s) return fail3(c, FDTD_ESTATE, "no 3D scene");
    if (comp < FDTD_EX || comp > FDTD_EZ) return fail3(c, FDTD_EINVAL, "3D sources drive Ex, Ey or Ez");
    const bool wall = (comp == FDTD_EX && (j < 1 || k < 1)) || (comp == FDTD_EY && (i < 1 || k < 1)) ||
                      (comp == FDTD_EZ && (i < 1 || j < 1));
    if (i < 0 || j < 0 || k < 0 || i >= s->nx || j >= s->ny || k >= s->nz || wall)
        return fail3(c, FDTD_EINVAL, "source (%d, %d, %d) outside the grid or on a PEC wall", i, j, k);
    if (kind < FDTD_SRC_RICKER || kind > FDTD_SRC_SINE) return fail3(c, FDTD_EINVAL, "unknown source kind");
    if (kind == FDTD_SRC_SAMPLED) {
        if (!samples || n_samples < 0) return fail3(c, FDTD_EINVAL, "sampled source needs samples");
        s->src_samples.assign(samples, samples + n_samples);
    } else {
        if (!params || !(params[0] > 0)) return fail3(c, FDTD_EINVAL, "source parameter must be > 0");
        s->src_param = params[0];
    }
    s->src_kind = kind; s->src_i = i; s->src_j = j; s->src_k = k; s->src_comp = comp;
    s->src_cap = 0;
    return FDTD_OK;
}

int fdtd_add_probe3(fdtd_ctx* c, int i, int j, int k, int comp, int* id) {
    Scene3* s = S3(c);
    if (!s) return fail3(c, FDTD_ESTATE, "no 3D scene");
    if (c->t != 0) return fail3(c, FDTD_ESTATE, "probes must be added before the first step");
    if (slot3(comp) < 0 || i < 0 || j < 0 || k < 0 || i >= s->nx || j >= s->ny || k >= s->nz)
        return fail3(c, FDTD_EINVAL, "bad probe");
    Sample3 sp{i, j, k, comp, (int)s->samples.size()};
    s->samples.push_back(sp);
    s->samp_dirty = true;
    if (s->d_rec) cudaFree(s->d_rec);
    s->d_rec = nullptr;
    s->rec_cap = 0;
    Probe p;
    p.scene = 0; p.slot = sp.slot; p.t_start = 0;
    c->probes.push_back(p);
    *id = (int)c->probes.size() - 1;
    return FDTD_OK;
}

int fdtd_add_dft_monitor3(fdtd_ctx* c, const int32_t* cells, int n_cells, const double* freqs, int n_freq, int* id) {
    Scene3* s = S3(c);
    if (!s) return fail3(c, FDTD_ESTATE, "no 3D scene");
    if (c->t != 0) return fail3(c, FDTD_ESTATE, "monitors must be added before the first step");
    if (!cells || n_cells < 1 || !freqs || n_freq < 1) return fail3(c, FDTD_EINVAL, "monitor needs cells and frequencies");
    DftMon m;
    m.scene = 0; m.n_cells = n_cells; m.n_freq = n_freq; m.slot0 = (int)s->samples.size();
    m.freqs.assign(freqs, freqs + n_freq);
    m.t_start = 0; m.plane_k = -1; m.comp_mask = 0; m.d_freq = nullptr; m.d_acc = nullptr;
    for (int q = 0; q < n_cells; q++) {
        const int i = cells[3 * q], j = cells[3 * q + 1], k = cells[3 * q + 2];
        if (i < 0 || j < 0 || k < 0 || i >= s->nx || j >= s->ny || k >= s->nz) return fail3(c, FDTD_EINVAL, "bad monitor cell");
    }
    if (cudaMalloc(&m.d_freq, n_freq * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&m.d_acc, (size_t)n_cells * n_freq * sizeof(float4)) != cudaSuccess) {
        cudaGetLastError();
        return fail3(c, FDTD_ENOMEM, "monitor");
    }
    CK3(cudaMemcpyAsync(m.d_freq, freqs, n_freq * sizeof(double), cudaMemcpyHostToDevice, c->stream), "monitor");
    CK3(cudaMemsetAsync(m.d_acc, 0, (size_t)n_cells * n_freq * sizeof(float4), c->stream), "monitor");
    CK3(cudaStreamSynchronize(c->stream), "monitor");
    for (int q = 0; q < n_cells; q++) {
        Sample3 sp{cells[3 * q], cells[3 * q + 1], cells[3 * q + 2], G_EZ, (int)s->samples.size()};
        s->samples.push_back(sp);
    }
    s->samp_dirty = true;
    if (s->d_rec) cudaFree(s->d_rec);
    s->d_rec = nullptr;
    s->rec_cap = 0;
    c->mons.push_back(m);
    *id = (int)c->mons.size() - 1;
    return FDTD_OK;
}

int fdtd_add_dft_plane3(fdtd_ctx* c, int k, int comp_mask, const double* freqs, int n_freq, int* id) {
    Scene3* s = S3(c);
    if (!s) return fail3(c, FDTD_ESTATE, "no 3D scene");
    if (c->t != 0) return fail3(c, FDTD_ESTATE, "monitors must be added before the first step");
    if (k < 0 || k >= s->nz || (comp_mask & ~7) || !comp_mask || !freqs || n_freq < 1 || n_freq > 16)
        return fail3(c, FDTD_EINVAL, "plane monitor: k in 0..nz-1, comp_mask of Ex|Ey|Ez bits, 1..16 frequencies");
    int ncomp = 0;
    for (int q = 0; q < 3; q++) ncomp += (comp_mask >> q) & 1;
    DftMon m;
    m.scene = 0; m.n_cells = s->nx * s->ny; m.n_freq = n_freq; m.slot0 = -1;
    m.freqs.assign(freqs, freqs + n_freq);
    m.t_start = 0; m.plane_k = k; m.comp_mask = comp_mask; m.d_freq = nullptr; m.d_acc = nullptr;
    const size_t bytes = (size_t)ncomp * n_freq * s->nx * s->ny * sizeof(float4);
    if (cudaMalloc(&m.d_freq, n_freq * sizeof(double)) != cudaSuccess || cudaMalloc(&m.d_acc, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail3(c, FDTD_ENOMEM, "plane monitor");
    }
    CK3(cudaMemcpyAsync(m.d_freq, freqs, n_freq * sizeof(double), cudaMemcpyHostToDevice, c->stream), "monitor");
    CK3(cudaMemsetAsync(m.d_acc, 0, bytes, c->stream), "monitor");
    CK3(cudaStreamSynchronize(c->stream), "monitor");
    c->mons.push_back(m);
    *id = (int)c->mons.size() - 1;
    return FDTD_OK;
}

// z-segments of the two-step kernel: [zb[b], zb[b + 1]).  Uniform segments of
// segz planes; with `align` and a CPML, the planes whose two-step footprint
// meets the z-slabs' reach get segments of their own at both ends, and the
// planes between are split evenly into segments of at most segz, so that the
// tiles there can run the build without the CPML.
static std::vector<int> z_bounds(int nz, int npml, int segz, bool align) {
    std::vector<int> zb{0};
    const int z1 = npml + 3, z2 = nz - npml - 2;   // [z1, z2): footprints clear of the z-slabs
    if (align && npml > 0 && z2 - z1 >= 1) {
        zb.push_back(z1);
        const int m = (z2 - z1 + segz - 1) / segz;
        for (int q = 1; q <= m; q++) zb.push_back(z1 + (int)((long long)(z2 - z1) * q / m));
        zb.push_back(nz);
    } else {
        for (int k = segz; k < nz; k += segz) zb.push_back(k);
        zb.push_back(nz);
    }
    return zb;
}

// samples by owning CTA of the two-step kernel's tiling (TX2 x T2_ROWS x the
// z-segments zb), the tile lists and the segment bounds on the device
static int build_s2(fdtd_ctx* c, Scene3* s, int key, const std::vector<int>& zb, const dim3& g2) {
    if (s->s2_seg == key) return FDTD_OK;
    const int ncta = (int)(g2.x * g2.y * g2.z);
    std::vector<int> cnt((size_t)ncta + 1, 0), idx(std::max<size_t>(1, s->samples.size()));
    auto seg_of = [&](int k) { return (int)(std::upper_bound(zb.begin(), zb.end(), k) - zb.begin()) - 1; };
    auto cta_of = [&](const Sample3& sp) {
        return (int)(sp.i / TX2 + g2.x * (sp.j / T2_ROWS + g2.y * seg_of(sp.k)));
    };
    for (const Sample3& sp : s->samples) cnt[cta_of(sp) + 1]++;
    for (int b = 0; b < ncta; b++) cnt[b + 1] += cnt[b];
    std::vector<int> pos(cnt.begin(), cnt.end() - 1);
    for (size_t q = 0; q < s->samples.size(); q++) idx[pos[cta_of(s->samples[q])]++] = (int)q;
    // a tile needs the CPML build when a lane, row or plane of its two-step
    // footprint meets the kernel's (conservative) CPML reach
    const int np = s->npml;
    auto reach = [&](int v, int n) { return v >= 0 && v < n && (v < np + 1 || v >= n - np - 1); };
    std::vector<int> tint, tpml;
    // the CPML build's x-slab lanes per warp: the most any x-tile has (the
    // kernel's own lane predicate)
    s->s2_xs = 1;
    if (np > 0)
        for (int bx = 0; bx < (int)g2.x; bx++) {
            int n = 0;
            for (int l = 0; l < 32; l++) {
                const int xc = bx * TX2 - 4 + 4 * l;
                n += (xc + 3 >= 0 && xc < s->nx && (xc - 1 < np + 1 || xc + 4 >= s->nx - np - 1)) ? 1 : 0;
            }
            s->s2_xs = std::max(s->s2_xs, n);
        }
    for (int t = 0; t < ncta; t++) {
        const int bx = t % (int)g2.x, by = (t / (int)g2.x) % (int)g2.y, bz = t / (int)(g2.x * g2.y);
        bool p = false;
        if (np > 0) {
            for (int l = 0; l < 32 && !p; l++) {
                const int xc = bx * TX2 - 4 + 4 * l;
                p = xc + 3 >= 0 && xc < s->nx && (xc - 1 < np + 1 || xc + 4 >= s->nx - np - 1);
            }
            for (int r = by * T2_ROWS - 2; r <= by * T2_ROWS + T2_ROWS && !p; r++) p = reach(r, s->ny);
            for (int k = zb[bz] - 2; k <= zb[bz + 1] && !p; k++) p = reach(k, s->nz);
        }
        (p ? tpml : tint).push_back(t);
    }
    s->n_s2int = (int)tint.size();
    s->n_s2pml = (int)tpml.size();
    tint.insert(tint.end(), tpml.begin(), tpml.end());
    if (s->d_s2off) cudaFree(s->d_s2off);
    if (s->d_s2idx) cudaFree(s->d_s2idx);
    if (s->d_s2tiles) cudaFree(s->d_s2tiles);
    if (s->d_s2zb) cudaFree(s->d_s2zb);
    s->d_s2off = s->d_s2idx = s->d_s2tiles = s->d_s2zb = nullptr;
    s->s2_seg = -1;
    if (cudaMalloc(&s->d_s2off, cnt.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&s->d_s2idx, idx.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&s->d_s2tiles, tint.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&s->d_s2zb, zb.size() * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail3(c, FDTD_ENOMEM, "tables of the two-step kernel");
    }
    if (!s->aux) {
        if (cudaStreamCreateWithFlags(&s->aux, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return fail3(c, FDTD_ECUDA, "second stream of the two-step kernel");
        }
    }
    CK3(cudaMemcpyAsync(s->d_s2off, cnt.data(), cnt.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream), "samples");
    CK3(cudaMemcpyAsync(s->d_s2idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream), "samples");
    CK3(cudaMemcpyAsync(s->d_s2tiles, tint.data(), tint.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream), "tiles");
    CK3(cudaMemcpyAsync(s->d_s2zb, zb.data(), zb.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream), "segments");
    CK3(cudaStreamSynchronize(c->stream), "samples");
    s->s2_seg = key;
    return FDTD_OK;
}

int fdtd_step3(fdtd_ctx* c, int64_t n_steps) {
    Scene3* s = S3(c);
    if (!s) return fail3(c, FDTD_ESTATE, "no 3D scene");
    int rc = ensure3(c, c->t + n_steps);
    if (rc) return rc;
    Dev3 d = dev_of(s);
    const dim3 blk(32, 8);
    const dim3 grd((s->nx + 31) / 32, (s->ny + 7) / 8, s->nz);
    const dim3 grp((s->nx + 31) / 32, (s->ny + 7) / 8, 1);
    const int si = s->src_kind >= 0 ? s->src_i : -1;
    // z-segment planes: the option, else 24 for the one-step kernel, 48 for the two-step one
    const int segz = c->opt_segment > 0 ? c->opt_segment : 24;
    const int seg2 = c->opt_segment > 0 ? c->opt_segment : 48;
    const dim3 gfz((s->nx + TXC - 1) / TXC, (s->ny + TYR - 1) / TYR, (s->nz + segz - 1) / segz);
    const size_t smem3 = fused3_smem();
    // the two-step kernel (FDTD_OPT_TBLOCK = 2) takes steps in pairs; it updates
    // at most MAXP2 plane monitors itself
    int n_plane = 0;
    for (const DftMon& m : c->mons) n_plane += m.plane_k >= 0 ? 1 : 0;
    bool two = c->opt_kernel != 1 && c->opt_tblock == 2 && n_plane <= MAXP2 && n_steps >= 2;
    // automatic segments are cut at the z-slabs' reach (see z_bounds)
    const std::vector<int> zb2 = z_bounds(s->nz, s->npml, seg2, c->opt_segment <= 0);
    const dim3 g2((s->nx + TX2 - 1) / TX2, (s->ny + T2_ROWS - 1) / T2_ROWS, (unsigned)zb2.size() - 1);
    const size_t smem2i = t2_smem<T2_ROWS, false>(0);
    if (c->opt_kernel != 1) {
        cudaError_t ea = ensure_dyn_smem((const void*)k_yee3d_fused, smem3);
        if (ea == cudaSuccess && two) ea = ensure_dyn_smem((const void*)k_yee3d_t2<T2_ROWS, false>, smem2i);
        if (ea != cudaSuccess) return fail3(c, FDTD_ECUDA, "fused 3D kernel: %s", cudaGetErrorString(ea));
    }
    size_t smem2p = 0;
    if (two) {
        rc = build_s2(c, s, 2 * seg2 + (c->opt_segment <= 0 ? 1 : 0), zb2, g2);
        if (rc) return rc;
        smem2p = t2_smem<T2_ROWS, true>(s->s2_xs);
        // a CPML so thick that a tile's slab lanes overflow shared memory: steps
        // run the one-step kernel
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (s->npml && smem2p > (size_t)optin) two = false;
    }
    if (two) {
        if (s->npml) {
            cudaError_t ea = ensure_dyn_smem((const void*)k_yee3d_t2<T2_ROWS, true>, smem2p);
            if (ea != cudaSuccess)
                return fail3(c, FDTD_ECUDA, "two-step 3D kernel, %zu B of shared memory (%d x-slab lanes per warp): %s",
                             smem2p, s->s2_xs, cudaGetErrorString(ea));
        }
        for (DftMon& m : c->mons)
            if (m.plane_k >= 0 && !m.d_e1) {
                const size_t b = (size_t)3 * s->rows * s->pitch * sizeof(float);
                if (cudaMalloc(&m.d_e1, b) != cudaSuccess) {
                    cudaGetLastError();
                    m.d_e1 = nullptr;
                    return fail3(c, FDTD_ENOMEM, "plane copy of the two-step kernel");
                }
            }
    }
    auto swap_bufs = [&]() {
        for (int w = 0; w < G_COUNT; w++) std::swap(s->f[w], s->g[w]);
        d = dev_of(s);
    };
    auto bufs = [&]() {
        Bufs3 b;
        for (int w = 0; w < G_COUNT; w++) {
            b.in[w] = s->f[w];
            b.out[w] = s->g[w];
        }
        return b;
    };
    // after step n: the source, probes and plane DFT (src_rec: the kernel has
    // not done them; pair: the plane DFT takes steps n - 1 and n, the first
    // from the two-step kernel's copy of the plane), then the cell monitors
    // from the record
    auto after = [&](long long n, bool src_rec, bool pair) {
        if (src_rec) {
            if (si >= 0 || !s->samples.empty()) {
                k_src_rec3<<<1, 128, 0, c->stream>>>(d, si, s->src_j, s->src_k, s->src_comp, s->d_src,
                                                     s->src_kind >= 0 ? s->src_cap : 0, s->d_samp,
                                                     (int)s->samples.size(), s->d_rec, n);
                c->launches++;
            }
        }
        for (const DftMon& m : c->mons) {
            if (m.plane_k >= 0) {
                if (!src_rec) continue;
                if (pair)
                    k_dft_plane3_pair<<<grp, blk, 0, c->stream>>>(d, m.plane_k, m.comp_mask, m.d_freq, m.n_freq, s->dt,
                                                                  m.d_acc, n - 1, m.d_e1);
                else
                    k_dft_plane3<<<grp, blk, 0, c->stream>>>(d, m.plane_k, m.comp_mask, m.d_freq, m.n_freq, s->dt,
                                                             m.d_acc, n);
            } else {
                k_dft_cells3<<<(m.n_cells * m.n_freq + 127) / 128, 128, 0, c->stream>>>(
                    s->d_rec, (int)s->samples.size(), m.slot0, m.n_cells, m.d_freq, m.n_freq, s->dt, m.d_acc, n);
            }
            c->launches++;
        }
    };
    for (int64_t q = 0; q < n_steps;) {
        const long long n = c->t + q;
        if (two && q + 1 < n_steps) {
            Extra2 x;
            memset(&x, 0, sizeof(x));
            x.wave = s->d_src;
            x.wlen = s->src_kind >= 0 ? s->src_cap : 0;
            x.si = si; x.sj = s->src_j; x.sk = s->src_k; x.scomp = s->src_comp - G_EX;
            x.samp = s->d_samp;
            x.n_samp = (int)s->samples.size();
            x.s_off = s->samples.empty() ? nullptr : s->d_s2off;
            x.s_idx = s->d_s2idx;
            x.rec = s->d_rec;
            for (const DftMon& m : c->mons)
                if (m.plane_k >= 0) {
                    x.mon_k[x.n_mon] = m.plane_k; x.mon_mask[x.n_mon] = m.comp_mask; x.mon_e1[x.n_mon] = m.d_e1;
                    x.n_mon++;
                }
            x.n = n;
            // tiles without CPML reach on the second stream, the others here
            const Bufs3 b2 = bufs();
            const int nthr = (T2_ROWS + 3) * 32;
            const bool fork = s->n_s2int > 0 && s->n_s2pml > 0;
            if (fork) {
                CK3(cudaEventRecord(s->ev_fork, c->stream), "fork");
                CK3(cudaStreamWaitEvent(s->aux, s->ev_fork, 0), "fork");
            }
            if (s->n_s2int > 0) {
                k_yee3d_t2<T2_ROWS, false><<<s->n_s2int, nthr, smem2i, fork ? s->aux : c->stream>>>(
                    d, b2, x, s->d_s2zb, s->d_s2tiles, (int)g2.x, (int)g2.y, 0);
                c->launches++;
            }
            if (s->n_s2pml > 0) {
                k_yee3d_t2<T2_ROWS, true><<<s->n_s2pml, nthr, smem2p, c->stream>>>(
                    d, b2, x, s->d_s2zb, s->d_s2tiles + s->n_s2int, (int)g2.x, (int)g2.y, s->s2_xs);
                c->launches++;
            }
            if (fork) {
                CK3(cudaEventRecord(s->ev_join, s->aux), "join");
                CK3(cudaStreamWaitEvent(c->stream, s->ev_join, 0), "join");
            }
            swap_bufs();
            after(n, false, false);
            after(n + 1, true, true);
            q += 2;
            continue;
        }
        if (c->opt_kernel == 1) {
            k_h3<<<grd, blk, 0, c->stream>>>(d);
            k_e3<<<grd, blk, 0, c->stream>>>(d);
            c->launches += 2;
        } else {
            k_yee3d_fused<<<gfz, NW3 * 32, smem3, c->stream>>>(d, bufs(), segz);
            c->launches++;
            swap_bufs();
        }
        after(n, true, false);
        q += 1;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail3(c, FDTD_ECUDA, "3D step: %s", cudaGetErrorString(e));
    c->t += n_steps;
    return FDTD_OK;
}

int fdtd_read_probe3(fdtd_ctx* c, int id, float* out, int64_t n) {
    Scene3* s = S3(c);
    if (id < 0 || id >= (int)c->probes.size()) return fail3(c, FDTD_EINVAL, "no probe %d", id);
    if (n < 0 || n > c->t) return fail3(c, FDTD_EINVAL, "asked for %lld samples, %lld recorded", (long long)n, (long long)c->t);
    if (n == 0) return FDTD_OK;
    const int nrec = (int)s->samples.size();
    CK3(cudaMemcpy2DAsync(out, sizeof(float), s->d_rec + c->probes[id].slot, (size_t)nrec * sizeof(float), sizeof(float),
                          (size_t)n, cudaMemcpyDeviceToHost, c->stream), "read probe");
    CK3(cudaStreamSynchronize(c->stream), "read probe");
    return FDTD_OK;
}

int fdtd_read_dft3(fdtd_ctx* c, int id, float* re, float* im) {
    if (id < 0 || id >= (int)c->mons.size()) return fail3(c, FDTD_EINVAL, "no monitor %d", id);
    const DftMon& m = c->mons[id];
    int ncomp = 1;
    if (m.plane_k >= 0) {
        ncomp = 0;
        for (int q = 0; q < 3; q++) ncomp += (m.comp_mask >> q) & 1;
    }
    const size_t n = (size_t)ncomp * m.n_freq * m.n_cells;
    std::vector<float4> acc(n);
    CK3(cudaMemcpyAsync(acc.data(), m.d_acc, n * sizeof(float4), cudaMemcpyDeviceToHost, c->stream), "read dft");
    CK3(cudaStreamSynchronize(c->stream), "read dft");
    for (size_t q = 0; q < n; q++) {
        re[q] = (float)((double)acc[q].x - (double)acc[q].z);
        im[q] = (float)((double)acc[q].y - (double)acc[q].w);
    }
    return FDTD_OK;
}

static cudaMemcpy3DParms copy3(const Scene3* s, float* dev_base, float* host, bool to_dev, bool on_device) {
    cudaMemcpy3DParms p;
    memset(&p, 0, sizeof(p));
    cudaPitchedPtr dp = make_cudaPitchedPtr(dev_base, (size_t)s->pitch * sizeof(float), s->pitch, s->rows);
    cudaPitchedPtr hp = make_cudaPitchedPtr(host, (size_t)s->nx * sizeof(float), s->nx, s->ny);
    const cudaPos dpos = make_cudaPos(PX3 * sizeof(float), 1, 1);
    const cudaPos hpos = make_cudaPos(0, 0, 0);
    if (to_dev) {
        p.srcPtr = hp; p.srcPos = hpos; p.dstPtr = dp; p.dstPos = dpos;
        p.kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    } else {
        p.srcPtr = dp; p.srcPos = dpos; p.dstPtr = hp; p.dstPos = hpos;
        p.kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    }
    p.extent = make_cudaExtent((size_t)s->nx * sizeof(float), s->ny, s->nz);
    return p;
}

int fdtd_get_field3(fdtd_ctx* c, int comp, float* out, int on_device) {
    Scene3* s = S3(c);
    const int q = slot3(comp);
    if (!s || q < 0) return fail3(c, FDTD_EINVAL, "bad component %d", comp);
    cudaMemcpy3DParms p = copy3(s, s->f[q], out, false, on_device != 0);
    CK3(cudaMemcpy3DAsync(&p, c->stream), "get field");
    CK3(cudaStreamSynchronize(c->stream), "get field");
    return FDTD_OK;
}

int fdtd_set_field3(fdtd_ctx* c, int comp, const float* in, int on_device) {
    Scene3* s = S3(c);
    const int q = slot3(comp);
    if (!s || q < 0) return fail3(c, FDTD_EINVAL, "bad component %d", comp);
    cudaMemcpy3DParms p = copy3(s, s->f[q], const_cast<float*>(in), true, on_device != 0);
    CK3(cudaMemcpy3DAsync(&p, c->stream), "set field");
    CK3(cudaStreamSynchronize(c->stream), "set field");
    return FDTD_OK;
}

int fdtd_reset3(fdtd_ctx* c) {
    Scene3* s = S3(c);
    const size_t n = (size_t)s->pitch * s->rows * s->planes * sizeof(float);
    for (int q = 0; q < G_COUNT; q++) {
        if (s->f[q]) CK3(cudaMemsetAsync(s->f[q], 0, n, c->stream), "reset");
        if (s->g[q]) CK3(cudaMemsetAsync(s->g[q], 0, n, c->stream), "reset");
    }
    if (s->d_rec) CK3(cudaMemsetAsync(s->d_rec, 0, (size_t)s->rec_cap * s->samples.size() * sizeof(float), c->stream), "reset");
    for (DftMon& m : c->mons) {
        int ncomp = 1;
        if (m.plane_k >= 0) {
            ncomp = 0;
            for (int q = 0; q < 3; q++) ncomp += (m.comp_mask >> q) & 1;
        }
        CK3(cudaMemsetAsync(m.d_acc, 0, (size_t)ncomp * m.n_freq * m.n_cells * sizeof(float4), c->stream), "reset");
    }
    CK3(cudaStreamSynchronize(c->stream), "reset");
    c->t = 0;
    return FDTD_OK;
}

int fdtd_save_state3(fdtd_ctx* c, void* buf, size_t* bytes) {
    Scene3* s = S3(c);
    const size_t n = (size_t)s->pitch * s->rows * s->planes * sizeof(float);
    int narr = 0;
    for (int q = 0; q < G_COUNT; q++) narr += s->f[q] ? 1 : 0;
    const size_t need = sizeof(int64_t) + (size_t)narr * n + (size_t)c->t * s->samples.size() * sizeof(float);
    if (!buf) {
        *bytes = need;
        return FDTD_OK;
    }
    if (*bytes < need) return fail3(c, FDTD_EINVAL, "state buffer too small");
    char* p = (char*)buf;
    memcpy(p, &c->t, sizeof(int64_t));
    p += sizeof(int64_t);
    for (int q = 0; q < G_COUNT; q++)
        if (s->f[q]) {
            CK3(cudaMemcpyAsync(p, s->f[q], n, cudaMemcpyDeviceToHost, c->stream), "save");
            p += n;
        }
    const size_t rb = (size_t)c->t * s->samples.size() * sizeof(float);
    if (rb) CK3(cudaMemcpyAsync(p, s->d_rec, rb, cudaMemcpyDeviceToHost, c->stream), "save");
    CK3(cudaStreamSynchronize(c->stream), "save");
    *bytes = need;
    return FDTD_OK;
}

int fdtd_load_state3(fdtd_ctx* c, const void* buf, size_t bytes) {
    Scene3* s = S3(c);
    if (bytes < sizeof(int64_t)) return fail3(c, FDTD_EINVAL, "state buffer too small");
    int64_t t;
    memcpy(&t, buf, sizeof(t));
    const size_t n = (size_t)s->pitch * s->rows * s->planes * sizeof(float);
    int narr = 0;
    for (int q = 0; q < G_COUNT; q++) narr += s->f[q] ? 1 : 0;
    const size_t need = sizeof(int64_t) + (size_t)narr * n + (size_t)t * s->samples.size() * sizeof(float);
    if (bytes < need) return fail3(c, FDTD_EINVAL, "state buffer too small");
    int rc = ensure3(c, std::max<int64_t>(t, 1));
    if (rc) return rc;
    const char* p = (const char*)buf + sizeof(int64_t);
    for (int q = 0; q < G_COUNT; q++)
        if (s->f[q]) {
            CK3(cudaMemcpyAsync(s->f[q], p, n, cudaMemcpyHostToDevice, c->stream), "load");
            p += n;
        }
    const size_t rb = (size_t)t * s->samples.size() * sizeof(float);
    if (rb) CK3(cudaMemcpyAsync(s->d_rec, p, rb, cudaMemcpyHostToDevice, c->stream), "load");
    CK3(cudaStreamSynchronize(c->stream), "load");
    c->t = t;
    return FDTD_OK;
}

int fdtd_check_finite3(fdtd_ctx* c) {
    Scene3* s = S3(c);
    int* d_bad = nullptr;
    if (cudaMalloc(&d_bad, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail3(c, FDTD_ENOMEM, "finite check");
    }
    cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream);
    const dim3 blk(32, 8);
    const dim3 grd((s->nx + 31) / 32, (s->ny + 7) / 8, s->nz);
    k_finite3<<<grd, blk, 0, c->stream>>>(dev_of(s), d_bad);
    c->launches++;
    int bad = 0;
    cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    cudaFree(d_bad);
    if (e != cudaSuccess) return fail3(c, FDTD_ECUDA, "finite check: %s", cudaGetErrorString(e));
    return bad ? fail3(c, FDTD_EUNSTABLE, "non-finite field values") : FDTD_OK;
}

}  // namespace gem

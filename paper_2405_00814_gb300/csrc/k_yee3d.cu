// 3D Yee path: the six-component extension of the leapfrog step that the paper
// says follows directly from the 2D scheme (Sec. II-B; Sec. III-A), with the same
// two layers (H from curl E, then E from curl H), per-cell Ca and Cb from eq. (7)
// for all three E components of a cell, and a CPML of twelve auxiliaries.
//
// Layout: every array is [nz + 2][ny + 2][pitch] FP32 with one zero pad cell on
// each side; cell (i, j, k) sits at ((k + 1)(ny + 2) + j + 1) pitch + i + 1, pitch
// = round_up(nx + 2, 32).  Tangential E on the walls i|j|k = 0 is never updated
// (stays zero); the pads are the ghost walls at N.  Fields are updated in place:
// one H launch and one E launch per step, then a small source/probe launch and
// the plane DFT.
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

// x offset of cell i = 0 in a row: a 4-float left pad keeps every 32-cell tile
// row 16-byte aligned for the fused kernel's staging
constexpr int PX3 = 4;

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
// fused z-marching step: one CTA owns a TX x TY tile of (i, j) and a z-segment
// [kA, kB).  Per plane k it stages E^n(k+1) with a one-cell halo in shared
// memory, updates H(k) on the tile plus its low halo (i0-1 column, j0-1 row,
// recomputed from the read-only input so no other CTA is waited on), then E(k)
// on the tile, with H(k-1) of its own column carried in registers.  Reads
// buffer `in`, writes buffer `out`.  A segment starting above k = 0 first
// recomputes H(kA-1) (warm-up plane, nothing stored).
// ---------------------------------------------------------------------------
constexpr int TX3 = 32, TY3 = 8;

struct Bufs3 {
    const float* in[G_COUNT];
    float* out[G_COUNT];
};

__device__ __forceinline__ void cpa16(float* smem, const float* gmem, bool valid) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(valid ? 16 : 0) : "memory");
}

constexpr int EW3 = 40;   // staged E row: storage columns [i0, i0 + 40) = cells i0 - 4 .. i0 + 35
constexpr int HW3 = 36;   // staged H row: cells i0 - 4 .. i0 + 31

__global__ void __launch_bounds__(TX3 * TY3) k_yee3d_fused(Dev3 S, Bufs3 B, int segz) {
    __shared__ __align__(16) float Eb[3][3][TY3 + 2][EW3];   // E^n, planes k, k+1, k+2 (ring by plane % 3)
    __shared__ __align__(16) float Hb[2][3][TY3 + 1][HW3];   // H^{n-1/2}, planes k, k+1 (ring by plane % 2)
    __shared__ float Ht[3][TY3 + 1][TX3 + 1];                // H^{n+1/2}(k) on the tile and its low halo
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX3 + tx;
    const int i0 = blockIdx.x * TX3, j0 = blockIdx.y * TY3;
    const int kA = blockIdx.z * segz, kB = min(kA + segz, S.nz);
    const size_t plane = (size_t)S.pitch * S.rows;
    // storage index of (column s of the staged row, row jj, plane k); column 0 is cell i0 - 4
    auto sidx = [&](int jj, int k) { return ((size_t)(k + 1) * S.rows + (jj + 1)) * S.pitch + i0; };
    const P3 pr{S.prof, S.pitch, S.rows, S.planes};
    const bool pml = S.has_pml != 0;
    const int i = i0 + tx, j = j0 + ty;
    const bool own = i < S.nx && j < S.ny;

    // staging: 16-byte copies of whole aligned row pieces; rows beyond the
    // padded array (jj > ny) and planes beyond nz read as zeros
    auto issue_e = [&](int k) {
        const int b = k % 3;
        for (int q = tid; q < 3 * (TY3 + 2) * (EW3 / 4); q += TX3 * TY3) {
            const int comp = q / ((TY3 + 2) * (EW3 / 4));
            const int r = q % ((TY3 + 2) * (EW3 / 4));
            const int qy = r / (EW3 / 4), v = r % (EW3 / 4);
            const int jj = j0 - 1 + qy;
            const bool in = jj <= S.ny && k <= S.nz;
            cpa16(&Eb[b][comp][qy][4 * v], B.in[G_EX + comp] + (in ? sidx(jj, k) + 4 * v : 0), in);
        }
    };
    auto issue_h = [&](int k) {
        const int b = k & 1;
        for (int q = tid; q < 3 * (TY3 + 1) * (HW3 / 4); q += TX3 * TY3) {
            const int comp = q / ((TY3 + 1) * (HW3 / 4));
            const int r = q % ((TY3 + 1) * (HW3 / 4));
            const int qy = r / (HW3 / 4), v = r % (HW3 / 4);
            const int jj = j0 - 1 + qy;
            const bool in = jj <= S.ny && k < S.nz;
            cpa16(&Hb[b][comp][qy][4 * v], B.in[G_HX + comp] + (in ? sidx(jj, k) + 4 * v : 0), in);
        }
    };

    // this thread's H cells (tile + low halo, (TY3+1) x (TX3+1) = 297 of them)
    // and their x/y CPML profiles, fixed for the whole march
    constexpr int NHC = ((TY3 + 1) * (TX3 + 1) + TX3 * TY3 - 1) / (TX3 * TY3);
    int hq[NHC], hqy[NHC], hqx[NHC];
    float hbx[NHC], hcx[NHC], hby[NHC], hcy[NHC];
#pragma unroll
    for (int u = 0; u < NHC; u++) {
        hq[u] = tid + u * TX3 * TY3;
        hqy[u] = hq[u] / (TX3 + 1);
        hqx[u] = hq[u] % (TX3 + 1);
        const int ii = i0 - 1 + hqx[u], jj = j0 - 1 + hqy[u];
        const bool ok = hq[u] < (TY3 + 1) * (TX3 + 1) && ii >= 0 && jj >= 0 && ii < S.nx && jj < S.ny;
        hbx[u] = ok && pml ? pr.bHx(ii + PX3) : 0.f;
        hcx[u] = ok && pml ? pr.cHx(ii + PX3) : 0.f;
        hby[u] = ok && pml ? pr.bHy(jj + 1) : 0.f;
        hcy[u] = ok && pml ? pr.cHy(jj + 1) : 0.f;
    }
    const float ebx = own && pml ? pr.bEx(i + PX3) : 0.f, ecx = own && pml ? pr.cEx(i + PX3) : 0.f;
    const float eby = own && pml ? pr.bEy(j + 1) : 0.f, ecy = own && pml ? pr.cEy(j + 1) : 0.f;

    const int kf = kA > 0 ? kA - 1 : 0;
    issue_e(kf);
    issue_e(kf + 1);
    issue_h(kf);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    float hx_prev = 0.f, hy_prev = 0.f;   // H(k-1) of this thread's column (zero pad below k = 0)
    const size_t own_row = ((size_t)(j + 1)) * S.pitch + (i + PX3);
    uint8_t m_next = own ? S.mat[(size_t)((kf < kA ? kA : kf) + 1) * plane + own_row] : 0;
    for (int k = kf; k < kB; k++) {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        // prefetch plane k+1's inputs while plane k computes (their slots held plane k-1)
        if (k + 1 < kB) {
            issue_e(k + 2);
            issue_h(k + 1);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        const uint8_t m_cur = m_next;
        if (own && k + 1 < kB) m_next = S.mat[(size_t)(k + 2) * plane + own_row];
        const int ec = k % 3, en = (k + 1) % 3, hb = k & 1;
        const float bz = pml ? pr.bHz(k + 1) : 0.f, cz = pml ? pr.cHz(k + 1) : 0.f;
        // ---- layer 1 on the tile and its low halo ----
#pragma unroll
        for (int u = 0; u < NHC; u++) {
            if (hq[u] >= (TY3 + 1) * (TX3 + 1)) break;
            const int qy = hqy[u], qx = hqx[u];
            const int ii = i0 - 1 + qx, jj = j0 - 1 + qy;
            float hx = 0.f, hy = 0.f, hz = 0.f;
            if (ii >= 0 && jj >= 0 && ii < S.nx && jj < S.ny) {
                const int sx = qx + 3;   // staged column of cell ii
                const size_t c = (size_t)(k + 1) * plane + (size_t)(jj + 1) * S.pitch + (ii + PX3);
                const float exc = Eb[ec][0][qy][sx], eyc = Eb[ec][1][qy][sx], ezc = Eb[ec][2][qy][sx];
                float dezy = Eb[ec][2][qy + 1][sx] - ezc;
                float deyz = Eb[en][1][qy][sx] - eyc;
                float dexz = Eb[en][0][qy][sx] - exc;
                float dezx = Eb[ec][2][qy][sx + 1] - ezc;
                float deyx = Eb[ec][1][qy][sx + 1] - eyc;
                float dexy = Eb[ec][0][qy + 1][sx] - exc;
                const bool owned = ii >= i0 && jj >= j0 && k >= kA;   // halo and warm-up values are not stored
                auto ps = [&](int slot, float bb, float cc, float d) {
                    if (bb == 0.f && cc == 0.f) return d;
                    const float vv = bb * B.in[slot][c] + cc * d;
                    if (owned) B.out[slot][c] = vv;
                    return d + vv;
                };
                if (pml) {
                    dezy = ps(P_HXY, hby[u], hcy[u], dezy);
                    deyz = ps(P_HXZ, bz, cz, deyz);
                    dexz = ps(P_HYZ, bz, cz, dexz);
                    dezx = ps(P_HYX, hbx[u], hcx[u], dezx);
                    deyx = ps(P_HZX, hbx[u], hcx[u], deyx);
                    dexy = ps(P_HZY, hby[u], hcy[u], dexy);
                }
                const int hx_ = qx + 3;
                hx = Hb[hb][0][qy][hx_] - (S.cdy * dezy - S.cdz * deyz);
                hy = Hb[hb][1][qy][hx_] - (S.cdz * dexz - S.cdx * dezx);
                hz = Hb[hb][2][qy][hx_] - (S.cdx * deyx - S.cdy * dexy);
                if (owned) {
                    B.out[G_HX][c] = hx;
                    B.out[G_HY][c] = hy;
                    B.out[G_HZ][c] = hz;
                }
            }
            Ht[0][qy][qx] = hx;
            Ht[1][qy][qx] = hy;
            Ht[2][qy][qx] = hz;
        }
        __syncthreads();
        // ---- layer 2 on the tile ----
        const float hxc = Ht[0][ty + 1][tx + 1], hyc = Ht[1][ty + 1][tx + 1], hzc = Ht[2][ty + 1][tx + 1];
        if (own && k >= kA) {
            const size_t c = (size_t)(k + 1) * plane + own_row;
            const float4 co = S.coef[m_cur];
            const float bez = pml ? pr.bEz(k + 1) : 0.f, cez = pml ? pr.cEz(k + 1) : 0.f;
            float dhzy = hzc - Ht[2][ty][tx + 1], dhyz = hyc - hy_prev;
            float dhxz = hxc - hx_prev, dhzx = hzc - Ht[2][ty + 1][tx];
            float dhyx = hyc - Ht[1][ty + 1][tx], dhxy = hxc - Ht[0][ty][tx + 1];
            const int sx = tx + 4;
            const float exc = Eb[ec][0][ty + 1][sx], eyc = Eb[ec][1][ty + 1][sx], ezc = Eb[ec][2][ty + 1][sx];
            auto ps = [&](int slot, float bb, float cc, float d) {
                if (bb == 0.f && cc == 0.f) return d;
                const float vv = bb * B.in[slot][c] + cc * d;
                B.out[slot][c] = vv;
                return d + vv;
            };
            float ex = exc, ey = eyc, ez = ezc;
            if (j >= 1 && k >= 1) {
                if (pml) {
                    dhzy = ps(P_EXY, eby, ecy, dhzy);
                    dhyz = ps(P_EXZ, bez, cez, dhyz);
                }
                ex = co.x * exc + co.z * dhzy - co.w * dhyz;
            }
            if (i >= 1 && k >= 1) {
                if (pml) {
                    dhxz = ps(P_EYZ, bez, cez, dhxz);
                    dhzx = ps(P_EYX, ebx, ecx, dhzx);
                }
                ey = co.x * eyc + co.w * dhxz - co.y * dhzx;
            }
            if (i >= 1 && j >= 1) {
                if (pml) {
                    dhyx = ps(P_EZX, ebx, ecx, dhyx);
                    dhxy = ps(P_EZY, eby, ecy, dhxy);
                }
                ez = co.x * ezc + co.y * dhyx - co.z * dhxy;
            }
            B.out[G_EX][c] = ex;
            B.out[G_EY][c] = ey;
            B.out[G_EZ][c] = ez;
        }
        hx_prev = hxc;
        hy_prev = hyc;
        __syncthreads();
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
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= S.nx || j >= S.ny) return;
    const size_t c = ((size_t)(plane_k + 1) * S.rows + (j + 1)) * S.pitch + (i + PX3);
    const size_t plane = (size_t)S.nx * S.ny;
    const size_t cell = (size_t)j * S.nx + i;
    const float fdt = (float)dt;
    int pc = 0;
    for (int comp = 0; comp < 3; comp++) {
        if (!(comp_mask & (1 << comp))) continue;
        const float e = S.f[comp][c];
        for (int f = 0; f < n_freq; f++) {
            double ph = freq[f] * dt * (double)(n + 1);
            ph -= floor(ph);
            double sn, cs;
            sincospi(2.0 * ph, &sn, &cs);
            float4 a = acc[((size_t)pc * n_freq + f) * plane + cell];
            kahan3(a.x, a.z, e * ((float)cs * fdt));
            kahan3(a.y, a.w, -e * ((float)sn * fdt));
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
    c->opt_kernel = 1; c->opt_tblock = 1; c->opt_segment = 64; c->opt_warps = 8;
    c->dirty = true;
    c->d_scenes = nullptr; c->d_tasks = nullptr; c->d_tasks_b = nullptr; c->n_tasks_b = 0; c->warps_b = 2; c->d_tasks_l = nullptr; c->n_tasks_l = 0; c->warps_l = 4;
    c->d_dft = nullptr; c->n_dft = 0; c->opt_adj_store = 1;
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
    s->nx = g->nx; s->ny = g->ny; s->nz = g->nz; s->npml = npml;
    s->dx = dx; s->dy = dy; s->dz = dz; s->dt = dt;
    s->pitch = (g->nx + PX3 + 40 + 31) / 32 * 32;   // room for the last tile's 40-float staging rows
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
    if (kind < FDTD_SRC_RICKER || kind > FDTD_SRC_SAMPLED) return fail3(c, FDTD_EINVAL, "unknown source kind");
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
    if (k < 0 || k >= s->nz || (comp_mask & ~7) || !comp_mask || !freqs || n_freq < 1)
        return fail3(c, FDTD_EINVAL, "plane monitor: k in 0..nz-1, comp_mask of Ex|Ey|Ez bits, frequencies");
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
    const int segz = std::max(1, c->opt_segment);
    const dim3 gfz((s->nx + TX3 - 1) / TX3, (s->ny + TY3 - 1) / TY3, (s->nz + segz - 1) / segz);
    for (int64_t q = 0; q < n_steps; q++) {
        const long long n = c->t + q;
        if (c->opt_kernel == 1) {
            k_h3<<<grd, blk, 0, c->stream>>>(d);
            k_e3<<<grd, blk, 0, c->stream>>>(d);
            c->launches += 2;
        } else {
            Bufs3 b;
            for (int w = 0; w < G_COUNT; w++) {
                b.in[w] = s->f[w];
                b.out[w] = s->g[w];
            }
            k_yee3d_fused<<<gfz, dim3(TX3, TY3), 0, c->stream>>>(d, b, segz);
            c->launches++;
            for (int w = 0; w < G_COUNT; w++) std::swap(s->f[w], s->g[w]);
            d = dev_of(s);
        }
        if (si >= 0 || !s->samples.empty()) {
            k_src_rec3<<<1, 128, 0, c->stream>>>(d, si, s->src_j, s->src_k, s->src_comp, s->d_src,
                                                 s->src_kind >= 0 ? s->src_cap : 0, s->d_samp, (int)s->samples.size(),
                                                 s->d_rec, n);
            c->launches++;
        }
        for (const DftMon& m : c->mons) {
            if (m.plane_k >= 0)
                k_dft_plane3<<<grp, blk, 0, c->stream>>>(d, m.plane_k, m.comp_mask, m.d_freq, m.n_freq, s->dt, m.d_acc, n);
            else
                k_dft_cells3<<<(m.n_cells * m.n_freq + 127) / 128, 128, 0, c->stream>>>(
                    s->d_rec, (int)s->samples.size(), m.slot0, m.n_cells, m.d_freq, m.n_freq, s->dt, m.d_acc, n);
            c->launches++;
        }
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

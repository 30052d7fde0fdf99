// One tile of one SSP-RK2 stage, shared by the plain (one tile per block)
// and fused (persistent, many tiles per block) kernels.
//
// A tile of cells is staged in shared memory with the stencil's halo: two
// cells on the upwind (low) side and one on the downwind side in every
// direction.  Every face value h = n_up + phi (n_dn - n_up)/2 is computed
// once into shared memory, then each cell takes the difference of its two
// faces per direction (Eq. 3 in semi-discrete flux form, SI Sec. S1.1):
//   STAGE 1: out = in + dt L(in)
//   STAGE 2: out = old/2 + (in + dt L(in))/2
// with L(n) = sum_d G_d (h_{d,-} - h_{d,+}) / dL_d plus the nucleation
// source B / (dL1 dL2) in the corner cell.  The volume moment (and, on
// output steps, all moments) of `out` accumulate into m[].
#pragma once

#include "pbe_device.cuh"

namespace pbe {

// The van Leer quotient q = b / (a + b) for a, b of the same strict sign,
// else 0 (the limited slope is then 2 a q, see Eq. 3), by the Newton-Raphson
// form: the hardware reciprocal approximation r ~ 1/s refined by one step on
// the quotient (q1 = q0 + r (b - s q0), error ~ (1 - s r)^2), and the
// same-sign test on the sign/exponent bits.  Faces where |a| or |b| is below
// 2^-959 are treated as flat (their limited slope is below 1e-288).
__device__ __forceinline__ double psi_quot_fast(double a, double b)
{
    const int ha = __double2hiint(a), hb = __double2hiint(b);
    const bool same = ((ha ^ hb) >= 0) && ((ha & 0x7ff00000) >= 0x04000000) && ((hb & 0x7ff00000) >= 0x04000000);
    double q = 0.0;
    if (same) {
        const double s = a + b;
        double rc;
        asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(rc) : "d"(s));
        const double q0 = b * rc;
        const double e = fma(-s, q0, b);
        q = fma(rc, e, q0);
    }
    return q;
}

// Half the van Leer limited slope, a q.
__device__ __forceinline__ double half_psi_fast(double a, double b) { return a * psi_quot_fast(a, b); }

// Face value n_up + psi/2 (FAST: one FMA on the quotient).
template <bool FAST>
__device__ __forceinline__ double face_value(double nm2, double up, double dn)
{
    if (FAST) {
        const double a = up - nm2;
        return fma(a, psi_quot_fast(a, dn - up), up);
    }
    return up + half_psi(up - nm2, dn - up);
}

template <bool CG>
__device__ __forceinline__ double ld_in(const double* p)
{
    return CG ? __ldcg(p) : *p;
}

// The 2-D moments of one cell value into m (order of the output rows) except
// the volume moment m[8], which the row kernels accumulate per column.
__device__ __forceinline__ void add_moments(double (&m)[10], double val, double x1, double x2, double area)
{
    const double w = val * area;
    const double x1w = x1 * w, x2w = x2 * w;
    m[0] += w; m[1] += x1w; m[2] += x2w;
    m[3] += x1 * x1w; m[4] += x1 * x2w; m[5] += x2 * x2w;
    m[6] += x1 * x1 * x1w; m[7] += x1 * x1 * x2w; m[9] += x2 * x2 * x2w;
}

// The sums over the 32 lanes of ten values, in the lanes (transposed
// butterfly: at offsets 16, 8, 4, 2 each lane keeps the lower or the upper
// part of its list, ceil(n/2) entries, and adds its partner's copy of it,
// then the pair at offset 1 adds).  Returns the total of value idx (lanes 2k
// and 2k+1 hold value k; idx >= 10 in the lanes that hold padding).  Twelve
// additions a lane against 310 in a lane-by-lane sum, in a fixed order.
__device__ __forceinline__ double transposed_sum10(const double (&v)[10], int lane, int& idx)
{
    const unsigned full = 0xffffffffu;
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    double w[5], x[3], y[2];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const double keep = b4 ? v[5 + i] : v[i], send = b4 ? v[i] : v[5 + i];
        w[i] = keep + __shfl_xor_sync(full, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const double hi = i + 3 < 5 ? w[i + 3] : 0.0;
        const double keep = b3 ? hi : w[i], send = b3 ? w[i] : hi;
        x[i] = keep + __shfl_xor_sync(full, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const double hi = i + 2 < 3 ? x[i + 2] : 0.0;
        const double keep = b2 ? hi : x[i], send = b2 ? x[i] : hi;
        y[i] = keep + __shfl_xor_sync(full, send, 4);
    }
    const double z = (b1 ? y[1] : y[0]) + __shfl_xor_sync(full, b1 ? y[0] : y[1], 2);
    // the kept entry's index, and whether it is a value or padding (real
    // entries of the kept list: 5 | 5, then 3 | 2 of five, 2 | 1 of three,
    // 1 | 1 of two; an upper part with fewer real entries is padded)
    int r = 5;
    r = b3 ? r - 3 : (r < 3 ? r : 3);
    r = b2 ? (r > 2 ? r - 2 : 0) : (r < 2 ? r : 2);
    r = b1 ? (r > 1 ? r - 1 : 0) : (r < 1 ? r : 1);
    idx = r > 0 ? (b4 ? 5 : 0) + (b3 ? 3 : 0) + (b2 ? 2 : 0) + (b1 ? 1 : 0) : 16;
    return z + __shfl_xor_sync(full, z, 1);
}

// Stage coefficients of one stage, uniform over the grid.
struct StageCoef {
    double c1, c2;   // G_d dt / dL_d
    double src;      // dt B / (dL1 dL2) (1-D: dt B / dL)
    bool moms;       // accumulate every moment (output step) or only the volume
};

// ---- 1-D -----------------------------------------------------------------
template <int STAGE, bool FAST, bool CG, int T, int NT>
__device__ __forceinline__ void tile1d(const double* in, const double* old, double* out, int i0, const Geom& g,
                                       const StageCoef& sc, double (&m)[4], double* tile, double* h)
{
    const int N = g.N1;
    for (int k = threadIdx.x; k < T + 3; k += NT) {
        int gi = i0 - 2 + k;
        tile[k] = (gi >= 0 && gi < N) ? ld_in<CG>(in + gi) : 0.0;
    }
    __syncthreads();
    // face f (0..T) lies between cells i0+f-1 (upwind) and i0+f
    for (int f = threadIdx.x; f <= T; f += NT) h[f] = face_value<FAST>(tile[f], tile[f + 1], tile[f + 2]);
    __syncthreads();
    for (int c = threadIdx.x; c < T; c += NT) {
        int i = i0 + c;
        if (i >= N) break;
        double v = tile[c + 2] + sc.c1 * (h[c] - h[c + 1]);
        if (i == 0) v += sc.src;
        if (STAGE == 2) v = 0.5 * old[i] + 0.5 * v;
        out[i] = v;
        double x = (i + 0.5) * g.d1;
        double w = v * g.d1;
        if (sc.moms) { m[0] += w; m[1] += x * w; m[2] += x * x * w; }
        m[3] += x * x * x * w;
    }
    __syncthreads();  // tile/h are reused by the next tile
}

// ---- 2-D -----------------------------------------------------------------
template <int TI, int TJ>
struct Tile2DSmem {
    double tile[(TI + 3) * (TJ + 3)];
    double h1[(TI + 1) * TJ];   // faces along L1: local face f between rows f-1 and f
    double h2[TI * (TJ + 1)];   // faces along L2
};

template <int STAGE, bool FAST, bool CG, int TI, int TJ, int NT>
__device__ __forceinline__ void tile2d(const double* in, const double* old, double* out, int i0, int j0,
                                       const Geom& g, const StageCoef& sc, double (&m)[10], Tile2DSmem<TI, TJ>& s)
{
    constexpr int W = TJ + 3;
    const int N1 = g.N1, N2 = g.N2;
    for (int k = threadIdx.x; k < (TI + 3) * W; k += NT) {
        int r = k / W, c = k - r * W;
        int gi = i0 - 2 + r, gj = j0 - 2 + c;
        s.tile[k] = (gi >= 0 && gi < N1 && gj >= 0 && gj < N2) ? ld_in<CG>(in + (size_t)gi * N2 + gj) : 0.0;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < (TI + 1) * TJ; k += NT) {
        int f = k / TJ, c = k - f * TJ;
        s.h1[k] = face_value<FAST>(s.tile[f * W + c + 2], s.tile[(f + 1) * W + c + 2], s.tile[(f + 2) * W + c + 2]);
    }
    for (int k = threadIdx.x; k < TI * (TJ + 1); k += NT) {
        int r = k / (TJ + 1), f = k - r * (TJ + 1);
        const double* row = s.tile + (r + 2) * W;
        s.h2[k] = face_value<FAST>(row[f], row[f + 1], row[f + 2]);
    }
    __syncthreads();
    const double area = g.d1 * g.d2;
    for (int k = threadIdx.x; k < TI * TJ; k += NT) {
        int r = k / TJ, c = k - r * TJ;
        int i = i0 + r, j = j0 + c;
        if (i >= N1 || j >= N2) continue;
        double v = s.tile[(r + 2) * W + c + 2] + sc.c1 * (s.h1[r * TJ + c] - s.h1[(r + 1) * TJ + c]) +
                   sc.c2 * (s.h2[r * (TJ + 1) + c] - s.h2[r * (TJ + 1) + c + 1]);
        if (i == 0 && j == 0) v += sc.src;
        size_t gidx = (size_t)i * N2 + j;
        if (STAGE == 2) v = 0.5 * old[gidx] + 0.5 * v;
        out[gidx] = v;
        double x1 = (i + 0.5) * g.d1, x2 = (j + 0.5) * g.d2;
        double w = v * area;
        double x1w = x1 * w, x2w = x2 * w;
        m[8] += x1 * x2 * x2w;
        if (sc.moms) {
            m[0] += w; m[1] += x1w; m[2] += x2w;
            m[3] += x1 * x1w; m[4] += x1 * x2w; m[5] += x2 * x2w;
            m[6] += x1 * x1 * x1w; m[7] += x1 * x1 * x2w; m[9] += x2 * x2 * x2w;
        }
    }
    __syncthreads();
}

// ---- split phases (used by the fused kernel to overlap the face work of the
// next stage with the scalar chain) -------------------------------------------
// Load a tile of the stage input with its halo and compute every face value.
// Runs on the `nthr` threads whose rank within the group is `tid`; `sync`
// synchronizes exactly those threads.
template <bool FAST, bool CG, int T, class Sync>
__device__ __forceinline__ void faces1d(const double* in, int i0, const Geom& g, double* tile, double* h, int tid,
                                        int nthr, Sync sync)
{
    const int N = g.N1;
    for (int k = tid; k < T + 3; k += nthr) {
        int gi = i0 - 2 + k;
        tile[k] = (gi >= 0 && gi < N) ? ld_in<CG>(in + gi) : 0.0;
    }
    sync();
    for (int f = tid; f <= T; f += nthr) h[f] = face_value<FAST>(tile[f], tile[f + 1], tile[f + 2]);
}

// Update the cells of a tile whose faces are in shared memory (all threads).
template <int STAGE, int T, int NT>
__device__ __forceinline__ void cells1d(const double* old, double* out, int i0, const Geom& g, const StageCoef& sc,
                                        double (&m)[4], const double* tile, const double* h)
{
    const int N = g.N1;
    for (int c = threadIdx.x; c < T; c += NT) {
        int i = i0 + c;
        if (i >= N) break;
        double v = tile[c + 2] + sc.c1 * (h[c] - h[c + 1]);
        if (i == 0) v += sc.src;
        if (STAGE == 2) v = 0.5 * old[i] + 0.5 * v;
        out[i] = v;
        double x = (i + 0.5) * g.d1;
        double w = v * g.d1;
        if (sc.moms) { m[0] += w; m[1] += x * w; m[2] += x * x * w; }
        m[3] += x * x * x * w;
    }
}

template <bool FAST, bool CG, int TI, int TJ, class Sync>
__device__ __forceinline__ void faces2d(const double* in, int i0, int j0, const Geom& g, Tile2DSmem<TI, TJ>& s,
                                        int tid, int nthr, Sync sync)
{
    constexpr int W = TJ + 3;
    const int N1 = g.N1, N2 = g.N2;
    for (int k = tid; k < (TI + 3) * W; k += nthr) {
        int r = k / W, c = k - r * W;
        int gi = i0 - 2 + r, gj = j0 - 2 + c;
        s.tile[k] = (gi >= 0 && gi < N1 && gj >= 0 && gj < N2) ? ld_in<CG>(in + (size_t)gi * N2 + gj) : 0.0;
    }
    sync();
    for (int k = tid; k < (TI + 1) * TJ; k += nthr) {
        int f = k / TJ, c = k - f * TJ;
        s.h1[k] = face_value<FAST>(s.tile[f * W + c + 2], s.tile[(f + 1) * W + c + 2], s.tile[(f + 2) * W + c + 2]);
    }
    for (int k = tid; k < TI * (TJ + 1); k += nthr) {
        int r = k / (TJ + 1), f = k - r * (TJ + 1);
        const double* row = s.tile + (r + 2) * W;
        s.h2[k] = face_value<FAST>(row[f], row[f + 1], row[f + 2]);
    }
}

template <int STAGE, int TI, int TJ, int NT>
__device__ __forceinline__ void cells2d(const double* old, double* out, int i0, int j0, const Geom& g,
                                        const StageCoef& sc, double (&m)[10], const Tile2DSmem<TI, TJ>& s)
{
    constexpr int W = TJ + 3;
    const int N1 = g.N1, N2 = g.N2;
    const double area = g.d1 * g.d2;
    for (int k = threadIdx.x; k < TI * TJ; k += NT) {
        int r = k / TJ, c = k - r * TJ;
        int i = i0 + r, j = j0 + c;
        if (i >= N1 || j >= N2) continue;
        double v = s.tile[(r + 2) * W + c + 2] + sc.c1 * (s.h1[r * TJ + c] - s.h1[(r + 1) * TJ + c]) +
                   sc.c2 * (s.h2[r * (TJ + 1) + c] - s.h2[r * (TJ + 1) + c + 1]);
        if (i == 0 && j == 0) v += sc.src;
        size_t gidx = (size_t)i * N2 + j;
        if (STAGE == 2) v = 0.5 * old[gidx] + 0.5 * v;
        out[gidx] = v;
        double x1 = (i + 0.5) * g.d1, x2 = (j + 0.5) * g.d2;
        double w = v * area;
        double x1w = x1 * w, x2w = x2 * w;
        m[8] += x1 * x2 * x2w;
        if (sc.moms) {
            m[0] += w; m[1] += x1w; m[2] += x2w;
            m[3] += x1 * x1w; m[4] += x1 * x2w; m[5] += x2 * x2w;
            m[6] += x1 * x1 * x1w; m[7] += x1 * x1 * x2w; m[9] += x2 * x2 * x2w;
        }
    }
}

template <int STAGE>
__device__ __forceinline__ StageCoef stage_coef(const Scal& S, const Geom& g)
{
    StageCoef sc;
    const double G1 = STAGE == 1 ? S.G1a : S.G1b;
    const double G2 = STAGE == 1 ? S.G2a : S.G2b;
    const double B = STAGE == 1 ? S.Ba : S.Bb;
    sc.c1 = G1 * S.dt / g.d1;
    sc.c2 = G2 * S.dt / g.d2;
    sc.src = g.ndim == 1 ? S.dt * B / g.d1 : S.dt * B / (g.d1 * g.d2);
    sc.moms = STAGE == 2 && S.clipped;
    return sc;
}

// The same with the reciprocal cell widths (one rounding more per product;
// used where one thread computes the coefficients for a whole block).
template <int STAGE>
__device__ __forceinline__ StageCoef stage_coef_fast(const Scal& S, const Geom& g)
{
    StageCoef sc;
    const double G1 = STAGE == 1 ? S.G1a : S.G1b;
    const double G2 = STAGE == 1 ? S.G2a : S.G2b;
    const double B = STAGE == 1 ? S.Ba : S.Bb;
    // (G / dL) dt: the rates per cell width are known before dt, so one
    // multiplication follows the step length
    sc.c1 = (G1 * g.inv_d1) * S.dt;
    sc.c2 = (G2 * g.inv_d2) * S.dt;
    sc.src = g.ndim == 1 ? (B * g.inv_d1) * S.dt : (B * (g.inv_d1 * g.inv_d2)) * S.dt;
    sc.moms = STAGE == 2 && S.clipped;
    return sc;
}

}  // namespace pbe

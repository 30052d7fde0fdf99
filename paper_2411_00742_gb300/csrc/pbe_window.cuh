// One window tile of one SSP-RK2 stage on a 2-D grid (the register-window
// layout of the split scheme's step kernel, for the unsplit stage of Eq. 3 in
// flux form), shared by the plain path's stage kernel and the fused path's
// persistent window kernel:
//   out = in + c1 (h1_{i-1/2} - h1_{i+1/2}) + c2 (h2_{j-1/2} - h2_{j+1/2})
//   (+ the nucleation inflow in cell (0, 0); stage 2 averages with n),
// both directions' faces from the same stage input.
//
// Block = 256 threads holding 128 consecutive columns j0-2 .. j0+125 of 2R
// rows and writing the 125 columns j0 .. j0+124:
//   1. L1 faces: every thread walks down its column (R rows) with a register
//      window of the input (2 rows above, 1 below), each face value once;
//      the input and the partial update w n + w c1 (h_up - h_dn) of every cell
//      go to shared memory (w = 1 in stage 1, 1/2 in stage 2, where the RK
//      average then adds n^k / 2);
//   2. L2 faces along the rows (8 warps x 2R/8 rows, four columns per lane):
//      both stencil differences of a face come from the lane or the lane
//      below, face values pass between lanes by shuffles; then the update and
//      the moments.
// Face quotients by the Newton-Raphson form (psi_quot_fast).
#pragma once

#include "pbe_tiles.cuh"

namespace pbe {

constexpr int kWNT = 256;             // threads per block
constexpr int kWX = 128;              // columns held per block
constexpr int kWOut = kWX - 3;        // columns written per block
constexpr int kWG = kWNT / kWX;       // row groups of the L1 pass
constexpr int kWW = kWNT / 32;        // warps
constexpr int kWC = kWX / 32;         // columns per lane in the L2 pass

// dynamic shared memory of a tile of R rows per group: the input and the partial update
constexpr size_t win_smem(int R) { return sizeof(double) * 2 * (kWG * R) * kWX; }

// Input loads: read-only cache in a stage kernel (CG false); L2 in the
// persistent kernel (CG true), whose input was written by other blocks of the
// same launch.
template <bool CG>
__device__ __forceinline__ double win_ld(const double* p)
{
    return CG ? __ldcg(p) : __ldg(p);
}

// The tile with origin (i0, j0) of stage STAGE.  Adds the tile's moments
// (all ten on output steps, sc.moms; else only the volume moment m[8]) to m.
// The moments are separable, mu_pq = sum_j x2_j^q dA sum_i x1_i^p n_ij: each
// lane sums S_p = sum_i x1_i^p n_ij down each of its four columns (three FMAs
// a cell beyond the volume moment's, instead of the ten moments a cell) and
// weights them with x2_j^q dA at the end of the tile.
// wsm: win_smem(kWR) bytes of dynamic shared memory; x1s: 3 kWG kWR doubles
// (x1, x1^2, x1^3 of the tile's rows).  MOMS: the caller's sc.moms, as a
// template argument so that the volume-only form carries no column sums.
// Starts and ends with the block's threads in step (one barrier between the
// passes); the caller separates consecutive tiles with a block barrier.
template <int STAGE, int kWR, bool CG, bool MOMS>
__device__ __forceinline__ void window_tile(const double* __restrict__ in, const double* old, double* out,
                                            const Geom& g, const StageCoef& sc, int i0, int j0, double* wsm,
                                            double* x1s, double (&m)[10])
{
    constexpr int kWTI = kWG * kWR;       // rows per block
    constexpr int kWRW = kWTI / kWW;      // rows per warp in the L2 pass
    double (*ins)[kWX] = reinterpret_cast<double (*)[kWX]>(wsm);              // stage input
    double (*f1s)[kWX] = reinterpret_cast<double (*)[kWX]>(wsm + kWTI * kWX); // w (in + c1 (h_up - h_dn))
    // stage 2 is n^k/2 + (n1 + dt L(n1))/2: the factor 1/2 goes into the coefficients
    constexpr double kW = STAGE == 2 ? 0.5 : 1.0;
    const double wc1 = kW * sc.c1, wc2 = kW * sc.c2, wsrc = kW * sc.src;
    const int N1 = g.N1, N2 = g.N2;
    if (threadIdx.x < kWTI) {
        const double x1 = (i0 + threadIdx.x + 0.5) * g.d1;
        x1s[threadIdx.x] = x1;
        if (MOMS) {
            x1s[kWTI + threadIdx.x] = x1 * x1;
            x1s[2 * kWTI + threadIdx.x] = x1 * x1 * x1;
        }
    }

    // 1. L1 faces down this thread's column: input rows i0+ra-2 .. i0+ra+kWR
    {
        const int tx = threadIdx.x % kWX, ra = (threadIdx.x / kWX) * kWR;
        const int j = j0 - 2 + tx;
        const bool jin = j >= 0 && j < N2;
        double v[kWR + 3];
#pragma unroll
        for (int q = 0; q < kWR + 3; ++q) {
            const int i = i0 + ra - 2 + q;
            v[q] = (jin && i >= 0 && i < N1) ? win_ld<CG>(in + (size_t)i * N2 + j) : 0.0;
        }
        const double a0 = v[1] - v[0];
        double dprev = v[2] - v[1];
        double hup = fma(a0, psi_quot_fast(a0, dprev), v[1]);   // face between rows i-1 and i
#pragma unroll
        for (int q = 0; q < kWR; ++q) {
            const double d = v[q + 3] - v[q + 2];
            const double hdn = fma(dprev, psi_quot_fast(dprev, d), v[q + 2]);   // face between rows i and i+1
            ins[ra + q][tx] = v[q + 2];
            f1s[ra + q][tx] = STAGE == 2 ? fma(wc1, hup - hdn, kW * v[q + 2]) : fma(wc1, hup - hdn, v[q + 2]);
            hup = hdn;
            dprev = d;
        }
    }
    __syncthreads();

    // 2. L2 faces, update and moments.  Local face c lies between columns c-1
    // and c; column c is updated from faces c and c+1.  Written columns:
    // local 2 .. kWX-2 (0, 1 and kWX-1 are halo).
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c0 = kWC * lane, jb = j0 - 2 + c0;
    const double area = g.d1 * g.d2;
    double acc[kWC], s0[kWC], s2[kWC], s3[kWC];   // S_1 (acc), S_0, S_2, S_3 of the lane's columns
    bool ok[kWC];
#pragma unroll
    for (int k = 0; k < kWC; ++k) {
        acc[k] = 0.0; s0[k] = 0.0; s2[k] = 0.0; s3[k] = 0.0;
        ok[k] = c0 + k >= 2 && c0 + k <= kWX - 2 && jb + k < N2;
    }
#pragma unroll
    for (int q = 0; q < kWRW; ++q) {
        const int r = warp * kWRW + q, i = i0 + r;
        const double2 p0 = *reinterpret_cast<const double2*>(&ins[r][c0]);
        const double2 p1 = *reinterpret_cast<const double2*>(&ins[r][c0 + 2]);
        const double c[kWC] = {p0.x, p0.y, p1.x, p1.y};
        const double cl = __shfl_up_sync(0xffffffffu, c[kWC - 1], 1);   // column c0-1
        double d[kWC];
        d[0] = c[0] - cl;
#pragma unroll
        for (int k = 1; k < kWC; ++k) d[k] = c[k] - c[k - 1];
        const double a0 = __shfl_up_sync(0xffffffffu, d[kWC - 1], 1);  // across face c0-1
        double h[kWC + 1];
        h[0] = fma(a0, psi_quot_fast(a0, d[0]), cl);
#pragma unroll
        for (int k = 1; k < kWC; ++k) h[k] = fma(d[k - 1], psi_quot_fast(d[k - 1], d[k]), c[k - 1]);
        h[kWC] = __shfl_down_sync(0xffffffffu, h[0], 1);                // face c0+kWC
        if (i >= N1) continue;
        const double2 f0 = *reinterpret_cast<const double2*>(&f1s[r][c0]);
        const double2 f1 = *reinterpret_cast<const double2*>(&f1s[r][c0 + 2]);
        const double fl[kWC] = {f0.x, f0.y, f1.x, f1.y};
        const size_t row = (size_t)i * N2;
        const double x1 = x1s[r];
#pragma unroll
        for (int k = 0; k < kWC; ++k) {
            if (!ok[k]) continue;
            double val = fma(wc2, h[k] - h[k + 1], fl[k]);
            if (i == 0 && jb + k == 0) val += wsrc;   // nucleation inflow, cell (0, 0)
            if (STAGE == 2) val = fma(0.5, CG ? __ldcg(old + row + jb + k) : old[row + jb + k], val);
            out[row + jb + k] = val;
            acc[k] = fma(x1, val, acc[k]);
            if (MOMS) {
                s0[k] += val;
                s2[k] = fma(x1s[kWTI + r], val, s2[k]);
                s3[k] = fma(x1s[2 * kWTI + r], val, s3[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kWC; ++k) {
        const double x2 = (jb + k + 0.5) * g.d2, a1 = x2 * area, a2 = x2 * a1;
        m[8] = fma(acc[k], a2, m[8]);
        if (MOMS) {   // mu_pq in row order; mu_12 (m[8]) above
            m[0] = fma(area, s0[k], m[0]); m[1] = fma(area, acc[k], m[1]); m[2] = fma(a1, s0[k], m[2]);
            m[3] = fma(area, s2[k], m[3]); m[4] = fma(a1, acc[k], m[4]); m[5] = fma(a2, s0[k], m[5]);
            m[6] = fma(area, s3[k], m[6]); m[7] = fma(a1, s2[k], m[7]); m[9] = fma(x2 * a2, s0[k], m[9]);
        }
    }
}

}  // namespace pbe

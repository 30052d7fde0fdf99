// The paper's scheme in 2-D: Eq. 3 (one-step high-resolution update with the
// van Leer limiter) with Godunov dimensional splitting, the L1 sweep then the
// L2 sweep, both in ONE kernel per step.
//
// In flux form with Courant number nu_d = G_d dt / dL_d per direction,
//   f_i <- f_i - nu (h_{i+1/2} - h_{i-1/2}),
//   h_{i+1/2} = f_i + (1 - nu) phi(theta_{i+1/2}) (f_{i+1} - f_i) / 2,
// which is Eq. 3 term by term (phi(theta) (f_{i+1} - f_i) = 2ab/(a+b) for
// a, b of the same strict sign, else 0).
//
// Block = 256 threads.  A block holds 128 consecutive columns j0-2 .. j0+125
// and writes the 125 columns j0 .. j0+124 of 32 rows:
//   1. L1 sweep (128 columns x 2 row groups of 16 rows): every thread walks
//      down its column with a register window of the input (2 rows above,
//      1 below), each face value computed once; the L1-swept values go to
//      shared memory;
//   2. L2 sweep along the rows (8 warps x 4 rows, four columns per lane):
//      both stencil differences of a face come from the lane itself or the
//      lane below, face values pass between lanes by shuffles; the three
//      extra columns are the stencil's halo, recomputed by the neighbouring
//      block;
//   3. update, nucleation inflow in the corner cell, the crystal-volume
//      moment (and every moment on output steps), last-block close of the
//      step: solute balance (Eq. 4), kinetics and CFL step of the next step.
// The state alternates between the two buffers with the parity of the step
// counter; launch_paper_finish copies it back after the last step.
//
// Face quotients use the Newton-Raphson form (half_psi_fast).  On GB300 the
// step is bound by the FP64 pipe: about 20 FP64 instructions per cell and
// step (per direction and face: one difference, five for the limited slope,
// one for the face value; two for the update; one for the volume moment)
// against 16 bytes of HBM traffic.
#include "pbe_internal.h"
#include "pbe_tiles.cuh"

namespace pbe {

constexpr int kPNT = 256;              // threads per block
constexpr int kPX = 128;               // columns held per block
constexpr int kPOut = kPX - 3;         // columns written per block
constexpr int kPG = kPNT / kPX;        // row groups of the L1 sweep
constexpr int kPR = 16;                // rows per row group
constexpr int kPTI = kPG * kPR;        // rows per block
constexpr int kPW = kPNT / 32;         // warps
constexpr int kPRW = kPTI / kPW;       // rows per warp in the L2 sweep
constexpr int kPC = kPX / 32;          // columns per lane in the L2 sweep

static inline int pdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

int paper_blocks2d(const Geom& g) { return pdiv(g.N2, kPOut) * pdiv(g.N1, kPTI); }

__global__ void __launch_bounds__(kPNT) k_lw_step2d(double* na, double* nb, Scal* S, Kin K, Geom g, double* part,
                                                     const double* t_out, double* rows, int use_cond,
                                                     cudaGraphConditionalHandle hcond)
{
    __shared__ __align__(16) double n1s[kPTI][kPX];
    __shared__ double x1s[kPTI];
    __shared__ double sh[kPW * 10];
    __shared__ int flag;
    if (S->done) {
        if (use_cond && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) cudaGraphSetConditional(hcond, 0);
        return;
    }
    const bool odd = (S->steps & 1) != 0;
    const double* __restrict__ in = odd ? nb : na;
    double* __restrict__ out = odd ? na : nb;
    const int N1 = g.N1, N2 = g.N2;
    const int i0 = blockIdx.y * kPTI, j0 = blockIdx.x * kPOut;
    const double dt = S->dt;
    const double nu1 = S->G1a * dt * g.inv_d1, om1 = 1.0 - nu1;
    const double nu2 = S->G2a * dt * g.inv_d2, om2 = 1.0 - nu2;
    const bool moms = S->clipped != 0;
    if (threadIdx.x < kPTI) x1s[threadIdx.x] = (i0 + threadIdx.x + 0.5) * g.d1;

    // 1. L1 sweep down this thread's column: input rows i0+ra-2 .. i0+ra+kPR
    {
        const int tx = threadIdx.x % kPX, ra = (threadIdx.x / kPX) * kPR;
        const int j = j0 - 2 + tx;
        const bool jin = j >= 0 && j < N2;
        double v[kPR + 3];
#pragma unroll
        for (int q = 0; q < kPR + 3; ++q) {
            const int i = i0 + ra - 2 + q;
            v[q] = (jin && i >= 0 && i < N1) ? __ldg(in + (size_t)i * N2 + j) : 0.0;
        }
        double dprev = v[2] - v[1];
        double hup = v[1] + om1 * half_psi_fast(v[1] - v[0], dprev);   // face between rows i-1 and i
#pragma unroll
        for (int q = 0; q < kPR; ++q) {
            const double d = v[q + 3] - v[q + 2];
            const double hdn = v[q + 2] + om1 * half_psi_fast(dprev, d);   // face between rows i and i+1
            n1s[ra + q][tx] = v[q + 2] + nu1 * (hup - hdn);
            hup = hdn;
            dprev = d;
        }
    }
    __syncthreads();

    // 2-3. L2 sweep, update and moments.  Local face c lies between columns
    // c-1 and c; column c is updated from faces c and c+1.  Written columns:
    // local 2 .. kPX-2 (0, 1 and kPX-1 are halo).
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c0 = kPC * lane, jb = j0 - 2 + c0;
    const double area = g.d1 * g.d2;
    double x2[kPC], acc[kPC];
    bool ok[kPC];
#pragma unroll
    for (int k = 0; k < kPC; ++k) {
        x2[k] = (jb + k + 0.5) * g.d2;
        acc[k] = 0.0;
        ok[k] = c0 + k >= 2 && c0 + k <= kPX - 2 && jb + k < N2;
    }
    double m[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) m[k] = 0.0;
    double v00 = 0.0;
#pragma unroll
    for (int q = 0; q < kPRW; ++q) {
        const int r = warp * kPRW + q, i = i0 + r;
        const double2 p0 = *reinterpret_cast<const double2*>(&n1s[r][c0]);
        const double2 p1 = *reinterpret_cast<const double2*>(&n1s[r][c0 + 2]);
        const double c[kPC] = {p0.x, p0.y, p1.x, p1.y};
        const double cl = __shfl_up_sync(0xffffffffu, c[kPC - 1], 1);   // column c0-1
        double d[kPC];
        d[0] = c[0] - cl;
#pragma unroll
        for (int k = 1; k < kPC; ++k) d[k] = c[k] - c[k - 1];
        const double a0 = __shfl_up_sync(0xffffffffu, d[kPC - 1], 1);  // across face c0-1
        double h[kPC + 1];
        h[0] = cl + om2 * half_psi_fast(a0, d[0]);
#pragma unroll
        for (int k = 1; k < kPC; ++k) h[k] = c[k - 1] + om2 * half_psi_fast(d[k - 1], d[k]);
        h[kPC] = __shfl_down_sync(0xffffffffu, h[0], 1);                // face c0+kPC
        if (i >= N1) continue;
        const size_t row = (size_t)i * N2;
        const double x1 = x1s[r];
#pragma unroll
        for (int k = 0; k < kPC; ++k) {
            const double val = c[k] + nu2 * (h[k] - h[k + 1]);
            if (q == 0 && k == 2) v00 = val;
            if (ok[k]) {
                out[row + jb + k] = val;
                acc[k] = fma(x1, val, acc[k]);
                if (moms) add_moments(m, val, x1, x2[k], area);
            }
        }
    }
    // nucleation inflow B dt / (dL1 dL2) into cell (0, 0): warp 0, lane 0, row 0, local column 2
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        const double src = dt * S->Ba / area;
        out[0] = v00 + src;
        acc[2] = fma(x1s[0], src, acc[2]);
        if (moms) add_moments(m, src, x1s[0], x2[2], area);
    }
    m[8] = 0.0;
#pragma unroll
    for (int k = 0; k < kPC; ++k) m[8] = fma(acc[k], x2[k] * x2[k] * area, m[8]);

    const int nbk = gridDim.x * gridDim.y, bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (moms) {
        block_sum<kPNT, 10>(m, sh);
        if (threadIdx.x == 0)
            for (int k = 0; k < 10; ++k) part[(size_t)bid * kMaxMom + k] = m[k];
    } else {
        double vv[1] = {m[8]};
        block_sum<kPNT, 1>(vv, sh);
        if (threadIdx.x == 0) part[(size_t)bid * kMaxMom + 8] = vv[0];
    }
    if (!last_block(&S->counter, nbk, &flag)) return;
    if (moms) {
        reduce_partials<kPNT, 10>(part, nbk, m, sh);
    } else {
        double vv[1];
        reduce_partials<kPNT, 1>(part + 8, nbk, vv, sh);
#pragma unroll
        for (int k = 0; k < 10; ++k) m[k] = 0.0;
        m[8] = vv[0];
    }
    if (threadIdx.x >= 32) return;
#pragma unroll
    for (int k = 0; k < 10; ++k) m[k] = __shfl_sync(0xffffffffu, m[k], 0);
    if (threadIdx.x == 0) S->counter = 0u;
    finish_stage2_warp(S, K, g, t_out, rows, m, 10, 8);
    if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(hcond, S->done ? 0u : 1u);
}

// After the last step: the state is in the second buffer when the number of
// steps taken is odd; copy it back.
__global__ void k_parity_fix(double* na, const double* nb, const Scal* S, long long ncell)
{
    if ((S->steps & 1) == 0) return;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x)
        na[c] = nb[c];
}

cudaError_t launch_paper_step2d(pbe_grid* g, bool use_cond, cudaGraphConditionalHandle h)
{
    const Geom& geo = g->geo;
    dim3 grid(pdiv(geo.N2, kPOut), pdiv(geo.N1, kPTI));
    k_lw_step2d<<<grid, kPNT, 0, g->stream>>>(g->d_n, g->d_n1, g->d_S, g->kin, geo, g->d_part, g->d_tout, g->d_rows,
                                               use_cond ? 1 : 0, h);
    return cudaGetLastError();
}

cudaError_t launch_paper_finish(pbe_grid* g)
{
    if (g->kin.scheme != PBE_SCHEME_PAPER || g->geo.ndim != 2) return cudaSuccess;
    const long long ncell = (long long)g->geo.N1 * g->geo.N2;
    long long nb = (ncell + 255) / 256;
    if (nb > 152 * 8) nb = 152 * 8;
    k_parity_fix<<<(int)nb, 256, 0, g->stream>>>(g->d_n, g->d_n1, g->d_S, ncell);
    return cudaGetLastError();
}

}  // namespace pbe

// Plain path, large 2-D grids: one SSP-RK2 stage per kernel with the
// register-window layout of the split scheme's step kernel (pbe_paper.cu),
// for the unsplit stage of Eq. 3 in flux form
//   out = in + c1 (h1_{i-1/2} - h1_{i+1/2}) + c2 (h2_{j-1/2} - h2_{j+1/2})
//   (+ the nucleation inflow in cell (0, 0); stage 2 averages with n),
// both directions' faces from the same stage input.
//
// Block = 256 threads holding 128 consecutive columns j0-2 .. j0+125 of 32
// rows and writing the 125 columns j0 .. j0+124:
//   1. L1 faces: every thread walks down its column (16 rows) with a register
//      window of the input (2 rows above, 1 below), each face value once;
//      the input and the partial update w n + w c1 (h_up - h_dn) of every cell
//      go to shared memory (w = 1 in stage 1, 1/2 in stage 2, where the RK
//      average then adds n^k / 2);
//   2. L2 faces along the rows (8 warps x 4 rows, four columns per lane): both
//      stencil differences of a face come from the lane or the lane below,
//      face values pass between lanes by shuffles; then the update, the
//      moments, and the last-block close of the stage (solute balance,
//      kinetics and step of the next stage) as in the tile kernels.
// Face quotients by the Newton-Raphson form (psi_quot_fast).  With 64 KB of
// shared memory and 4000 cells a block, the kernel is used when the grid
// gives at least one block per SM; smaller grids keep the tile kernels.
#include "pbe_internal.h"
#include "pbe_tiles.cuh"

namespace pbe {

constexpr int kWNT = 256;             // threads per block
constexpr int kWX = 128;              // columns held per block
constexpr int kWOut = kWX - 3;        // columns written per block
constexpr int kWG = kWNT / kWX;       // row groups of the L1 pass
constexpr int kWW = kWNT / 32;        // warps
constexpr int kWC = kWX / 32;         // columns per lane in the L2 pass
// rows per row group R (a block holds 2R rows, each warp 2R/8 of them in the
// L2 pass): 12, 16 or 20, chosen per grid so that the blocks spread evenly
// over the SMs (the kernel is bound by each SM's FP64 pipe)
constexpr size_t win_smem(int R) { return sizeof(double) * 2 * (kWG * R) * kWX; }   // input and partial update

static inline int wdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

static int window_blocks_r(const Geom& g, int R) { return wdiv(g.N2, kWOut) * wdiv(g.N1, kWG * R); }

int window_blocks2d(const Geom& g) { return window_blocks_r(g, 16); }

// the R whose block count divides most evenly into the SMs (blocks / (SMs x
// the most blocks any SM runs)); ties keep 16
static int window_rows(const Geom& g, int sms)
{
    int best = 16;
    double best_bal = 0.0;
    for (int R : {16, 12, 20}) {
        const int nb = window_blocks_r(g, R);
        const double bal = (double)nb / ((double)wdiv(nb, sms) * sms);
        if (bal > best_bal + 1e-9) { best_bal = bal; best = R; }
    }
    return best;
}

bool use_window2d(const pbe_grid* g)
{
    if (g->geo.ndim != 2 || g->window_mode == 0) return false;
    return g->window_mode == 1 || window_blocks2d(g->geo) >= g->sms;
}

template <int STAGE, int kWR>
__global__ void __launch_bounds__(kWNT) k_stage2d_win(const double* __restrict__ in, const double* old, double* out,
                                                     Scal* S, Kin K, Geom g, double* part, const double* t_out,
                                                     double* rows, int use_cond, cudaGraphConditionalHandle hcond)
{
    constexpr int kWTI = kWG * kWR;       // rows per block
    constexpr int kWRW = kWTI / kWW;      // rows per warp in the L2 pass
    extern __shared__ __align__(16) double wsm[];
    double (*ins)[kWX] = reinterpret_cast<double (*)[kWX]>(wsm);              // stage input
    double (*f1s)[kWX] = reinterpret_cast<double (*)[kWX]>(wsm + kWTI * kWX); // w (in + c1 (h_up - h_dn))
    __shared__ double x1s[kWTI];
    __shared__ double sh[kWW * 10];
    __shared__ int flag;
    if (S->done) {
        if (STAGE == 2 && use_cond && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
            cudaGraphSetConditional(hcond, 0);
        return;
    }
    StageCoef sc = stage_coef_fast<STAGE>(*S, g);
    if (K.kind == PBE_KINETICS_MLP) sc.moms = true;   // the closure reads mu0 at every stage
    // stage 2 is n^k/2 + (n1 + dt L(n1))/2: the factor 1/2 goes into the coefficients
    constexpr double kW = STAGE == 2 ? 0.5 : 1.0;
    const double wc1 = kW * sc.c1, wc2 = kW * sc.c2, wsrc = kW * sc.src;
    const int N1 = g.N1, N2 = g.N2;
    const int i0 = blockIdx.y * kWTI, j0 = blockIdx.x * kWOut;
    if (threadIdx.x < kWTI) x1s[threadIdx.x] = (i0 + threadIdx.x + 0.5) * g.d1;

    // 1. L1 faces down this thread's column: input rows i0+ra-2 .. i0+ra+kWR
    {
        const int tx = threadIdx.x % kWX, ra = (threadIdx.x / kWX) * kWR;
        const int j = j0 - 2 + tx;
        const bool jin = j >= 0 && j < N2;
        double v[kWR + 3];
#pragma unroll
        for (int q = 0; q < kWR + 3; ++q) {
            const int i = i0 + ra - 2 + q;
            v[q] = (jin && i >= 0 && i < N1) ? __ldg(in + (size_t)i * N2 + j) : 0.0;
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
    double x2[kWC], acc[kWC];
    bool ok[kWC];
#pragma unroll
    for (int k = 0; k < kWC; ++k) {
        x2[k] = (jb + k + 0.5) * g.d2;
        acc[k] = 0.0;
        ok[k] = c0 + k >= 2 && c0 + k <= kWX - 2 && jb + k < N2;
    }
    double m[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) m[k] = 0.0;
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
            if (STAGE == 2) val = fma(0.5, old[row + jb + k], val);
            out[row + jb + k] = val;
            acc[k] = fma(x1, val, acc[k]);
            if (sc.moms) add_moments(m, val, x1, x2[k], area);
        }
    }
#pragma unroll
    for (int k = 0; k < kWC; ++k) m[8] = fma(acc[k], x2[k] * x2[k] * area, m[8]);

    const int nb = gridDim.x * gridDim.y, bid = blockIdx.y * gridDim.x + blockIdx.x;
    block_sum<kWNT, 10>(m, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 10; ++k) part[(size_t)bid * kMaxMom + k] = m[k];
    if (!last_block(&S->counter, nb, &flag)) return;
    reduce_partials<kWNT, 10>(part, nb, m, sh);
    if (threadIdx.x >= 32) return;
#pragma unroll
    for (int k = 0; k < 10; ++k) m[k] = __shfl_sync(0xffffffffu, m[k], 0);
    if (threadIdx.x == 0) S->counter = 0u;
    if (STAGE == 1) {
        finish_stage1_warp(S, K, m[8], m[0]);
    } else {
        finish_stage2_warp(S, K, g, t_out, rows, m, 10, 8);
        if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(hcond, S->done ? 0u : 1u);
    }
}

template <int R>
static cudaError_t window_setup_r()
{
    cudaError_t e = cudaFuncSetAttribute(k_stage2d_win<1, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)win_smem(R));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_stage2d_win<2, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)win_smem(R));
    return e;
}

cudaError_t window_setup()
{
    cudaError_t e = window_setup_r<12>();
    if (e == cudaSuccess) e = window_setup_r<16>();
    if (e == cudaSuccess) e = window_setup_r<20>();
    return e;
}

template <int R>
static void launch_window_r(pbe_grid* g, int stage, int uc, cudaGraphConditionalHandle h)
{
    const Geom& geo = g->geo;
    const dim3 grid(wdiv(geo.N2, kWOut), wdiv(geo.N1, kWG * R));
    if (stage == 1)
        k_stage2d_win<1, R><<<grid, kWNT, win_smem(R), g->stream>>>(g->d_n, g->d_n, g->d_n1, g->d_S, g->kin, geo,
                                                                   g->d_part, g->d_tout, g->d_rows, uc, h);
    else
        k_stage2d_win<2, R><<<grid, kWNT, win_smem(R), g->stream>>>(g->d_n1, g->d_n, g->d_n, g->d_S, g->kin, geo,
                                                                   g->d_part, g->d_tout, g->d_rows, uc, h);
}

cudaError_t launch_window_stage2d(pbe_grid* g, int stage, bool use_cond, cudaGraphConditionalHandle h)
{
    const int uc = use_cond ? 1 : 0;
    switch (window_rows(g->geo, g->sms)) {
        case 12: launch_window_r<12>(g, stage, uc, h); break;
        case 20: launch_window_r<20>(g, stage, uc, h); break;
        default: launch_window_r<16>(g, stage, uc, h); break;
    }
    return cudaGetLastError();
}

}  // namespace pbe

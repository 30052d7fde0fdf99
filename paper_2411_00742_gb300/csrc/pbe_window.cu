// Plain path, large 2-D grids: one SSP-RK2 stage per kernel in the
// register-window layout (the tile body is window_tile, pbe_window.cuh), then
// the moments and the last-block close of the stage (solute balance, kinetics
// and step of the next stage) as in the tile kernels.  With 64 KB of shared
// memory and 4000 cells a block, the kernel is used when the grid gives at
// least one block per SM; smaller grids keep the tile kernels.
//
// Fused path, the same grids: one persistent cooperative launch per solve
// (k_fused_win) whose blocks loop over window tiles, the stages separated by
// the device-wide barrier that sums the volume moment (barrier_sum), every
// block advancing its own copy of the scalar chain (fused_finish*).
#include "pbe_chain.cuh"
#include "pbe_internal.h"
#include "pbe_sync.cuh"
#include "pbe_window.cuh"

#include <algorithm>

namespace pbe {

// rows per row group R (a block holds 2R rows, each warp 2R/8 of them in the
// L2 pass): 12, 16 or 20, chosen per grid so that the blocks spread evenly
// over the SMs (the kernel is bound by each SM's FP64 pipe)
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
    extern __shared__ __align__(16) double wsm[];
    __shared__ double x1s[3 * kWG * kWR];
    __shared__ double sh[kWW * 10];
    __shared__ int flag;
    if (S->done) {
        if (STAGE == 2 && use_cond && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
            cudaGraphSetConditional(hcond, 0);
        return;
    }
    StageCoef sc = stage_coef_fast<STAGE>(*S, g);
    if (K.kind == PBE_KINETICS_MLP) sc.moms = true;   // the closure reads mu0 at every stage
    double m[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) m[k] = 0.0;
    if (sc.moms) window_tile<STAGE, kWR, false, true>(in, old, out, g, sc, blockIdx.y * kWG * kWR, blockIdx.x * kWOut, wsm, x1s, m);
    else window_tile<STAGE, kWR, false, false>(in, old, out, g, sc, blockIdx.y * kWG * kWR, blockIdx.x * kWOut, wsm, x1s, m);

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

// Fused path, large 2-D grids: the whole solve in one cooperative launch.
// Each block owns an even contiguous share of the window tiles (tile t:
// rows (t / tiles_x) 2R.., columns (t % tiles_x) 125..) and runs them every
// stage, so a cell's stage-2 base value is read back by the thread that wrote
// it; halo rows and columns written by other blocks are read through L2
// (window_tile<.., CG = true>) after the device-wide barrier of the stage,
// which also sums the volume moment in fixed point (barrier_sum).  Warp 0 of
// every block then advances the block's copy of the scalar chain
// (fused_finish1/2, identical in every block).  Output steps: every block's
// ten moments go to rowpart, summed per row after the solve (k_fused_rows).
// Same parameters as k_fused; ti = rows per tile.
template <int kWR>
__global__ void __launch_bounds__(kWNT, 2) k_fused_win(double* n, double* n1, Scal* S, Kin K, Geom g, double* part,
                                                      const double* t_out, double* rows, unsigned int* bar,
                                                      int ntiles, int tiles_x, int ti, long long wait_limit,
                                                      double* rowpart)
{
    constexpr int NM = 10, VIDX = 8;
    constexpr int kWTI = kWG * kWR;
    extern __shared__ __align__(16) double wsm[];
    __shared__ double x1s[3 * kWTI];
    __shared__ Scal s;
    __shared__ StageCoef scs;
    __shared__ double red[kWW * NM];
    __shared__ long long wsum[kWW];
    __shared__ double msum[NM];
    __shared__ int fail;
    (void)part;
    (void)ti;
    if (threadIdx.x == 0) {
        s = *S;
        s.row_first = s.out_idx;   // rows before this index came from the prologue
        scs = stage_coef_fast<1>(s, g);
        fail = 0;
    }
    if (threadIdx.x < NM) msum[threadIdx.x] = 0.0;
    __syncthreads();
    if (s.done) {
        if (blockIdx.x == 0 && threadIdx.x == 0) S->row_first = s.row_first;
        return;
    }
    const int G = gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* my_rows = blockIdx.x == 0 ? rows : nullptr;
    // fixed-point unit of the volume-moment sum, as in k_fused
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(bar);
    unsigned long long acc_base0 = 0ull, acc_base1 = 0ull;
    double u, inv_u;
    {
        double vmax = 2.0 * (s.V0 + (K.kappa > 0.0 ? s.C / K.kappa : 0.0));
        if (!(vmax > 0.0) || !isfinite(vmax)) vmax = 1.0;
        const int E = ilogb(vmax) + 1;
        u = ldexp(1.0, E - 52);
        inv_u = ldexp(1.0, 52 - E);
    }
    unsigned int gen = 0;
    // warp 0: the stage-1 chain's evaluation, for the stage-2 chain's series
    // (in shared memory: the kernel's registers are at the 2-blocks-per-SM limit)
    __shared__ RateCarry rcs[32];
    if (warp == 0) rate_carry_init(rcs[lane], K);
    const int t_first = (int)(((long long)blockIdx.x * ntiles) / G);
    const int t_end = (int)(((long long)(blockIdx.x + 1) * ntiles) / G);
    for (;;) {
        KinT tpre{0.0, 0.0};
        if (warp == 0 && K.kind != PBE_KINETICS_FIXED) tpre = kin_temperature(K, s.t_new);
#pragma unroll 1
        for (int stage = 1; stage <= 2; ++stage) {
            const StageCoef sc = scs;
            double m[NM];
#pragma unroll
            for (int k = 0; k < NM; ++k) m[k] = 0.0;
            for (int t = t_first; t < t_end; ++t) {
                const int i0 = (t / tiles_x) * kWTI, j0 = (t % tiles_x) * kWOut;
                if (stage == 1) {
                    if (sc.moms) window_tile<1, kWR, true, true>(n, n, n1, g, sc, i0, j0, wsm, x1s, m);
                    else window_tile<1, kWR, true, false>(n, n, n1, g, sc, i0, j0, wsm, x1s, m);
                } else {
                    if (sc.moms) window_tile<2, kWR, true, true>(n1, n, n, g, sc, i0, j0, wsm, x1s, m);
                    else window_tile<2, kWR, true, false>(n1, n, n, g, sc, i0, j0, wsm, x1s, m);
                }
                __syncthreads();
            }
            const int row_here = s.out_idx;
            if (sc.moms) {   // the warp's ten moments (transposed butterfly), then over the warps
                int idx;
                const double tot = transposed_sum10(m, lane, idx);
                if ((lane & 1) == 0 && idx < NM) red[warp * NM + idx] = tot;
            }
            const long long qb = block_sum_fixed_t0(m[VIDX], inv_u, wsum);   // its barrier orders red
            if (sc.moms && threadIdx.x < NM) {
                double v = 0.0;
#pragma unroll
                for (int w = 0; w < kWW; ++w) v += red[w * NM + threadIdx.x];
                rowpart[((size_t)row_here * G + blockIdx.x) * NM + threadIdx.x] = v;
            }
            if (warp == 0) {
                if (threadIdx.x == 0) {
                    double total = 0.0;
                    const int p = (int)(gen & 1u);
                    unsigned long long base = p ? acc_base1 : acc_base0;
                    const bool ok = barrier_sum(acc + p * kAccStride, base, qb, u, (unsigned int)G, wait_limit, total);
                    if (p) acc_base1 = base;
                    else acc_base0 = base;
                    msum[VIDX] = total;
                    fail = !ok;
                }
                __syncwarp();
                if (!fail) {
                    const StageCoef c = stage == 1 ? fused_finish1<false, true>(&s, K, g, msum[VIDX], tpre, &rcs[lane])
                                                   : fused_finish2<false, true>(&s, K, g, t_out, my_rows, msum, NM, VIDX, tpre, &rcs[lane]);
                    if (threadIdx.x == 0) scs = c;
                }
            }
            gen += 1u;
            __syncthreads();
            if (fail || s.done) break;
        }
        if (s.done || fail) break;
    }
    if (threadIdx.x == 0 && fail) {
        S->status = PBE_ETIMEOUT;
        S->done = 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && !fail) {
        s.counter = 0u;
        *S = s;
    }
}

// Configuration of the fused window launch of a 2-D grid: the R (rows per
// group) with the least work on the busiest SM, estimated as the tiles per SM
// times the rows a tile loads (2R + 3, halo included); blocks = the
// co-resident ones, at most one per tile and max_blocks.
cudaError_t fused_window_config(const Geom& g, int sms, int max_blocks, FusedWinCfg* c)
{
    double best = 1e300;
    for (int R : {16, 12, 20}) {
        const void* fn = R == 12 ? (const void*)k_fused_win<12> : R == 20 ? (const void*)k_fused_win<20>
                                                                         : (const void*)k_fused_win<16>;
        const size_t dyn = win_smem(R);
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kWNT, dyn);
        if (e != cudaSuccess) return e;
        if (occ < 1) continue;
        const int tiles_x = wdiv(g.N2, kWOut), ntiles = tiles_x * wdiv(g.N1, kWG * R);
        int G = std::min(ntiles, occ * sms);
        G = std::min(G, max_blocks);
        G = std::min(G, 1000);   // the arrival count of barrier_sum has 10 bits
        const double cost = (double)wdiv(ntiles, sms) * (2 * R + 3);
        if (cost < best - 1e-9) {
            best = cost;
            c->fn = fn;
            c->dyn = dyn;
            c->G = G < 1 ? 1 : G;
            c->ntiles = ntiles;
            c->tiles_x = tiles_x;
            c->ti = kWG * R;
        }
    }
    return best < 1e300 ? cudaSuccess : cudaErrorInvalidConfiguration;
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

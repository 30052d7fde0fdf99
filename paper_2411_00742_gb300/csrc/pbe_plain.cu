// Plain path: one kernel per SSP-RK2 stage.  Each kernel stages a tile of
// the distribution with its 2-cell upwind / 1-cell downwind halo in shared
// memory, computes every face value once, updates its cells, and reduces
// the crystal-volume moment; the last block to finish closes the solute
// balance (Eq. 4) and evaluates the kinetics of the next stage on the
// device, so no scalar ever travels to the host between stages.
#include "pbe_internal.h"
#include "pbe_tiles.cuh"

namespace pbe {

constexpr int kNT = 256;      // threads per block
constexpr int kT1 = 1024;     // 1-D tile (cells per block)
constexpr int kTI = 16;       // 2-D tile rows (L1)
constexpr int kTJ = 32;       // 2-D tile columns (L2, contiguous)

static inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

int plain_max_blocks(const Geom& g)
{
    if (g.ndim == 1) return cdiv(g.N1, kT1);
    return cdiv(g.N1, kTI) * cdiv(g.N2, kTJ);
}

__global__ void k_set_scalars(Scal* S, double C, double t)
{
    S->C = C;
    S->t = t;
    S->V0 = 0.0;
    S->steps = 0;
    S->done = 1;
    S->status = 0;
    S->out_idx = 0;
    S->n_out = 0;
    S->counter = 0u;
}

// ---------------------------------------------------------------------------
// moments of the current state; prologue of a solve (or plain read-out)
// ---------------------------------------------------------------------------
template <int NDIM>
__global__ void __launch_bounds__(kNT) k_prologue(const double* __restrict__ n, Scal* S, Kin K, Geom g,
                                                  double* part, const double* t_out, double* rows,
                                                  int n_out, long long max_steps, double* mom_out)
{
    constexpr int NM = NDIM == 1 ? 4 : 10;
    constexpr int VIDX = NDIM == 1 ? 3 : 8;
    __shared__ double sh[kNT / 32 * NM];
    __shared__ int flag;
    double m[NM];
#pragma unroll
    for (int k = 0; k < NM; ++k) m[k] = 0.0;
    const int nb = gridDim.x;
    const long long ncell = (long long)g.N1 * g.N2;
    for (long long c = (long long)blockIdx.x * kNT + threadIdx.x; c < ncell; c += (long long)nb * kNT) {
        if (NDIM == 1) {
            double x = (c + 0.5) * g.d1;
            double v = n[c] * g.d1;
            m[0] += v; m[1] += x * v; m[2] += x * x * v; m[3] += x * x * x * v;
        } else {
            int i = (int)(c / g.N2), j = (int)(c % g.N2);
            double x1 = (i + 0.5) * g.d1, x2 = (j + 0.5) * g.d2;
            double v = n[c] * g.d1 * g.d2;
            double x1v = x1 * v, x2v = x2 * v;
            m[0] += v; m[1] += x1v; m[2] += x2v;
            m[3] += x1 * x1v; m[4] += x1 * x2v; m[5] += x2 * x2v;
            m[6] += x1 * x1 * x1v; m[7] += x1 * x1 * x2v; m[8] += x1 * x2 * x2v; m[9] += x2 * x2 * x2v;
        }
    }
    block_sum<kNT, NM>(m, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < NM; ++k) part[(size_t)blockIdx.x * kMaxMom + k] = m[k];
    if (!last_block(&S->counter, nb, &flag)) return;
    reduce_partials<kNT, NM>(part, nb, m, sh);
    if (threadIdx.x >= 32) return;
#pragma unroll
    for (int k = 0; k < NM; ++k) m[k] = __shfl_sync(0xffffffffu, m[k], 0);
    if (threadIdx.x == 0) {
        S->counter = 0u;
        if (mom_out) {  // read-out only
            for (int k = 0; k < NM; ++k) mom_out[k] = m[k];
        } else {
            S->V0 = m[VIDX];
            S->M0 = m[0];
            S->steps = 0;
            S->status = 0;
            S->done = 0;
            S->out_idx = 0;
            S->n_out = n_out;
            S->max_steps = max_steps;
            bool finite = isfinite(S->C) && isfinite(S->t);
            for (int k = 0; k < NM; ++k) finite = finite && isfinite(m[k]);
            if (!finite) {
                S->status = PBE_ENONFINITE;
                S->done = 1;
            } else {
                while (S->out_idx < n_out && t_out[S->out_idx] == S->t) {
                    double* row = rows + (size_t)S->out_idx * (NM + 2);
                    row[0] = S->t;
                    for (int k = 0; k < NM; ++k) row[1 + k] = m[k];
                    row[NM + 1] = S->C;
                    S->out_idx += 1;
                }
                if (S->out_idx >= n_out) S->done = 1;
            }
        }
    }
    __syncwarp();
    if (mom_out || S->done) return;
    prepare_step_warp(S, K, g, t_out);
}

// ---------------------------------------------------------------------------
// stage kernels: one tile per block, the last block closes the stage
//   STAGE 1: n1 = n + dt L(n; G_a, B_a)
//   STAGE 2: n  = n/2 + (n1 + dt L(n1; G_b, B_b))/2   (in place)
// ---------------------------------------------------------------------------
template <int STAGE>
__global__ void __launch_bounds__(kNT) k_stage1d(const double* __restrict__ in, const double* old, double* out,
                                                 Scal* S, Kin K, Geom g, double* part, const double* t_out,
                                                 double* rows, int use_cond, cudaGraphConditionalHandle hcond)
{
    __shared__ double tile[kT1 + 3];
    __shared__ double h[kT1 + 1];
    __shared__ double sh[kNT / 32 * 4];
    __shared__ int flag;
    if (S->done) {
        if (STAGE == 2 && use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(hcond, 0);
        return;
    }
    StageCoef sc = stage_coef<STAGE>(*S, g);
    if (K.kind == PBE_KINETICS_MLP) sc.moms = true;   // the closure reads mu0 at every stage
    double m[4] = {0.0, 0.0, 0.0, 0.0};
    tile1d<STAGE, true, false, kT1, kNT>(in, old, out, blockIdx.x * kT1, g, sc, m, tile, h);
    block_sum<kNT, 4>(m, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) part[(size_t)blockIdx.x * kMaxMom + k] = m[k];
    if (!last_block(&S->counter, gridDim.x, &flag)) return;
    reduce_partials<kNT, 4>(part, gridDim.x, m, sh);
    if (threadIdx.x >= 32) return;
#pragma unroll
    for (int k = 0; k < 4; ++k) m[k] = __shfl_sync(0xffffffffu, m[k], 0);
    if (threadIdx.x == 0) S->counter = 0u;
    if (STAGE == 1) {
        finish_stage1_warp(S, K, m[3], m[0]);
    } else {
        finish_stage2_warp(S, K, g, t_out, rows, m, 4, 3);
        if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(hcond, S->done ? 0u : 1u);
    }
}

template <int STAGE>
__global__ void __launch_bounds__(kNT) k_stage2d(const double* __restrict__ in, const double* old, double* out,
                                                 Scal* S, Kin K, Geom g, double* part, const double* t_out,
                                                 double* rows, int use_cond, cudaGraphConditionalHandle hcond)
{
    __shared__ Tile2DSmem<kTI, kTJ> ts;
    __shared__ double sh[kNT / 32 * 10];
    __shared__ int flag;
    if (S->done) {
        if (STAGE == 2 && use_cond && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
            cudaGraphSetConditional(hcond, 0);
        return;
    }
    const int nb = gridDim.x * gridDim.y, bid = blockIdx.y * gridDim.x + blockIdx.x;
    StageCoef sc = stage_coef<STAGE>(*S, g);
    if (K.kind == PBE_KINETICS_MLP) sc.moms = true;   // the closure reads mu0 at every stage
    double m[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) m[k] = 0.0;
    tile2d<STAGE, false, false, kTI, kTJ, kNT>(in, old, out, blockIdx.y * kTI, blockIdx.x * kTJ, g, sc, m, ts);
    block_sum<kNT, 10>(m, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 10; ++k) part[(size_t)bid * kMaxMom + k] = m[k];
    if (!last_block(&S->counter, nb, &flag)) return;
    reduce_partials<kNT, 10>(part, nb, m, sh);
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

// ---------------------------------------------------------------------------
// The paper's scheme in 1-D: Eq. 3 (one-step high-resolution update, van
// Leer limiter); the 2-D split form is in pbe_paper.cu.  With Courant number
// nu = G dt / dL, f_i <- f_i - nu (h_{i+1/2} - h_{i-1/2}),
// h_{i+1/2} = f_i + (1 - nu) phi(theta_{i+1/2}) (f_{i+1} - f_i) / 2.
// ---------------------------------------------------------------------------
// 1-D: the sweep (n -> n1), then a close kernel that copies n1 back to n with
// the nucleation inflow, the moments and the last-block close of the step.
__global__ void __launch_bounds__(kNT) k_sweep1d(const double* __restrict__ in, double* out, const Scal* S, Geom g)
{
    __shared__ double tile[kT1 + 3];
    __shared__ double h[kT1 + 1];
    if (S->done) return;
    const int N = g.N1, i0 = blockIdx.x * kT1;
    const double dt = S->dt, nu = S->G1a * dt / g.d1, om = 1.0 - nu;
    for (int k = threadIdx.x; k < kT1 + 3; k += kNT) {
        int gi = i0 - 2 + k;
        tile[k] = (gi >= 0 && gi < N) ? in[gi] : 0.0;
    }
    __syncthreads();
    for (int f = threadIdx.x; f <= kT1; f += kNT) {
        const double up = tile[f + 1];
        h[f] = up + om * half_psi(up - tile[f], tile[f + 2] - up);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < kT1; c += kNT) {
        int i = i0 + c;
        if (i >= N) break;
        out[i] = tile[c + 2] + nu * (h[c] - h[c + 1]);
    }
}

__global__ void __launch_bounds__(kNT) k_close1d(const double* __restrict__ in, double* out, Scal* S, Kin K, Geom g,
                                                 double* part, const double* t_out, double* rows, int use_cond,
                                                 cudaGraphConditionalHandle hcond)
{
    __shared__ double sh[kNT / 32 * 4];
    __shared__ int flag;
    if (S->done) {
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(hcond, 0);
        return;
    }
    const int N = g.N1;
    const double dt = S->dt;
    const bool moms = S->clipped;
    double m[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = blockIdx.x * kNT + threadIdx.x; i < N; i += gridDim.x * kNT) {
        double v = in[i];
        if (i == 0) v += dt * S->Ba / g.d1;
        out[i] = v;
        double x = (i + 0.5) * g.d1, w = v * g.d1;
        if (moms) { m[0] += w; m[1] += x * w; m[2] += x * x * w; }
        m[3] += x * x * x * w;
    }
    block_sum<kNT, 4>(m, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) part[(size_t)blockIdx.x * kMaxMom + k] = m[k];
    if (!last_block(&S->counter, gridDim.x, &flag)) return;
    reduce_partials<kNT, 4>(part, gridDim.x, m, sh);
    if (threadIdx.x >= 32) return;
#pragma unroll
    for (int k = 0; k < 4; ++k) m[k] = __shfl_sync(0xffffffffu, m[k], 0);
    if (threadIdx.x == 0) S->counter = 0u;
    finish_stage2_warp(S, K, g, t_out, rows, m, 4, 3);
    if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(hcond, S->done ? 0u : 1u);
}

// ---------------------------------------------------------------------------
// Gaussian seed: the density exp(-q/2) sampled at the cell centres (q the
// squared Mahalanobis distance of the normal with the given means, standard
// deviations and correlation).  Block sums of the density and of its volume
// moment weight (x^3 in 1-D, x1 x2^2 in 2-D) go to part[] for the scaling.
// ---------------------------------------------------------------------------
template <int NDIM>
__global__ void __launch_bounds__(kNT) k_seed_pdf(double* n, Geom g, double m1, double m2, double s1, double s2,
                                                  double rho, double* part)
{
    __shared__ double sh[kNT / 32 * 2];
    const long long ncell = (long long)g.N1 * g.N2;
    double acc[2] = {0.0, 0.0};
    for (long long c = (long long)blockIdx.x * kNT + threadIdx.x; c < ncell; c += (long long)gridDim.x * kNT) {
        double q, wv;
        if (NDIM == 1) {
            const double x = (c + 0.5) * g.d1;
            const double z = (x - m1) / s1;
            q = z * z;
            wv = x * x * x;
        } else {
            const int i = (int)(c / g.N2), j = (int)(c % g.N2);
            const double x1 = (i + 0.5) * g.d1, x2 = (j + 0.5) * g.d2;
            const double z1 = (x1 - m1) / s1, z2 = (x2 - m2) / s2;
            q = (z1 * z1 - 2.0 * rho * z1 * z2 + z2 * z2) / (1.0 - rho * rho);
            wv = x1 * x2 * x2;
        }
        const double f = exp(-0.5 * q);
        n[c] = f;
        acc[0] += f;
        acc[1] += wv * f;
    }
    block_sum<kNT, 2>(acc, sh);
    if (threadIdx.x == 0) {
        part[(size_t)blockIdx.x * kMaxMom] = acc[0];
        part[(size_t)blockIdx.x * kMaxMom + 1] = acc[1];
    }
}

__global__ void __launch_bounds__(kNT) k_seed_total(const double* part, int nb, double* total)
{
    __shared__ double sh[kNT / 32 * 2];
    double v[2];
    reduce_partials<kNT, 2>(part, nb, v, sh);
    if (threadIdx.x == 0) {
        total[0] = v[0];
        total[1] = v[1];
    }
}

__global__ void k_scale(double* n, long long ncell, double a)
{
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x)
        n[c] *= a;
}

cudaError_t launch_seed_pdf(pbe_grid* g, const double* mean, const double* sd, double corr, double* total_dev)
{
    const long long ncell = (long long)g->geo.N1 * g->geo.N2;
    int nb = cdiv(ncell, kNT);
    if (nb > 1024) nb = 1024;
    if (g->geo.ndim == 1)
        k_seed_pdf<1><<<nb, kNT, 0, g->stream>>>(g->d_n, g->geo, mean[0], 0.0, sd[0], 1.0, 0.0, g->d_part);
    else
        k_seed_pdf<2><<<nb, kNT, 0, g->stream>>>(g->d_n, g->geo, mean[0], mean[1], sd[0], sd[1], corr, g->d_part);
    k_seed_total<<<1, kNT, 0, g->stream>>>(g->d_part, nb, total_dev);
    return cudaGetLastError();
}

cudaError_t launch_scale(pbe_grid* g, double a)
{
    const long long ncell = (long long)g->geo.N1 * g->geo.N2;
    int nb = cdiv(ncell, kNT);
    if (nb > 4096) nb = 4096;
    k_scale<<<nb, kNT, 0, g->stream>>>(g->d_n, ncell, a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_set_scalars(pbe_grid* g, double C, double t)
{
    k_set_scalars<<<1, 1, 0, g->stream>>>(g->d_S, C, t);
    return cudaGetLastError();
}

cudaError_t launch_prologue(pbe_grid* g, int n_out, long long max_steps, double* mom_out)
{
    long long ncell = (long long)g->geo.N1 * g->geo.N2;
    int nb = cdiv(ncell, kNT);
    if (nb > g->max_blocks) nb = g->max_blocks;
    if (nb < 1) nb = 1;
    if (g->geo.ndim == 1)
        k_prologue<1><<<nb, kNT, 0, g->stream>>>(g->d_n, g->d_S, g->kin, g->geo, g->d_part, g->d_tout,
                                                 g->d_rows, n_out, max_steps, mom_out);
    else
        k_prologue<2><<<nb, kNT, 0, g->stream>>>(g->d_n, g->d_S, g->kin, g->geo, g->d_part, g->d_tout,
                                                 g->d_rows, n_out, max_steps, mom_out);
    return cudaGetLastError();
}

cudaError_t launch_plain_stage(pbe_grid* g, int stage)
{
    const Geom& geo = g->geo;
    if (geo.ndim == 1) {
        int nb = cdiv(geo.N1, kT1);
        if (stage == 1)
            k_stage1d<1><<<nb, kNT, 0, g->stream>>>(g->d_n, g->d_n, g->d_n1, g->d_S, g->kin, geo, g->d_part,
                                                    g->d_tout, g->d_rows, 0, 0);
        else
            k_stage1d<2><<<nb, kNT, 0, g->stream>>>(g->d_n1, g->d_n, g->d_n, g->d_S, g->kin, geo, g->d_part,
                                                    g->d_tout, g->d_rows, 0, 0);
    } else if (use_window2d(g)) {
        return launch_window_stage2d(g, stage, false, 0);
    } else {
        dim3 grid(cdiv(geo.N2, kTJ), cdiv(geo.N1, kTI));
        if (stage == 1)
            k_stage2d<1><<<grid, kNT, 0, g->stream>>>(g->d_n, g->d_n, g->d_n1, g->d_S, g->kin, geo, g->d_part,
                                                      g->d_tout, g->d_rows, 0, 0);
        else
            k_stage2d<2><<<grid, kNT, 0, g->stream>>>(g->d_n1, g->d_n, g->d_n, g->d_S, g->kin, geo, g->d_part,
                                                      g->d_tout, g->d_rows, 0, 0);
    }
    return cudaGetLastError();
}

cudaError_t launch_plain_step(pbe_grid* g, bool use_cond, cudaGraphConditionalHandle h)
{
    const Geom& geo = g->geo;
    int uc = use_cond ? 1 : 0;
    if (g->kin.scheme == PBE_SCHEME_PAPER) {
        if (geo.ndim == 1) {
            int nb = cdiv(geo.N1, kT1);
            k_sweep1d<<<nb, kNT, 0, g->stream>>>(g->d_n, g->d_n1, g->d_S, geo);
            int nc = cdiv(geo.N1, kNT);
            if (nc > g->max_blocks) nc = g->max_blocks;
            k_close1d<<<nc, kNT, 0, g->stream>>>(g->d_n1, g->d_n, g->d_S, g->kin, geo, g->d_part, g->d_tout,
                                                 g->d_rows, uc, h);
            return cudaGetLastError();
        }
        return launch_paper_step2d(g, use_cond, h);
    }
    if (geo.ndim == 1) {
        int nb = cdiv(geo.N1, kT1);
        k_stage1d<1><<<nb, kNT, 0, g->stream>>>(g->d_n, g->d_n, g->d_n1, g->d_S, g->kin, geo, g->d_part,
                                                g->d_tout, g->d_rows, uc, h);
        k_stage1d<2><<<nb, kNT, 0, g->stream>>>(g->d_n1, g->d_n, g->d_n, g->d_S, g->kin, geo, g->d_part,
                                                g->d_tout, g->d_rows, uc, h);
    } else if (use_window2d(g)) {
        cudaError_t e = launch_window_stage2d(g, 1, use_cond, h);
        if (e == cudaSuccess) e = launch_window_stage2d(g, 2, use_cond, h);
        return e;
    } else {
        dim3 grid(cdiv(geo.N2, kTJ), cdiv(geo.N1, kTI));
        k_stage2d<1><<<grid, kNT, 0, g->stream>>>(g->d_n, g->d_n, g->d_n1, g->d_S, g->kin, geo, g->d_part,
                                                  g->d_tout, g->d_rows, uc, h);
        k_stage2d<2><<<grid, kNT, 0, g->stream>>>(g->d_n1, g->d_n, g->d_n, g->d_S, g->kin, geo, g->d_part,
                                                  g->d_tout, g->d_rows, uc, h);
    }
    return cudaGetLastError();
}

}  // namespace pbe

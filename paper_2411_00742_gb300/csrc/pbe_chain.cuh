// The scalar chain between the two stages of a step, arranged for the
// latency of one warp (used by the persistent kernels): the solute balance
// of Eq. 4, the kinetics, the CFL step and the next stage's coefficients.
#pragma once

#include "pbe_tiles.cuh"

namespace pbe {

// finite and nonzero, on the bits (integer operations)
__device__ __forceinline__ bool finite_nonzero_bits(double x)
{
    const long long b = __double_as_longlong(x);
    return (b & 0x7ff0000000000000LL) != 0x7ff0000000000000LL && (b & 0x7fffffffffffffffLL) != 0;
}

// The stage-2 rates of a step from its stage-1 rates.  Both chains evaluate
// the kinetics at the step's end time (the same solubility c* and Arrhenius
// factor), so for the power law, with d = C - c*,
//   G(d) = G(d0) (1 + delta)^p,  delta = (d - d0) / d0,
// and (1 + delta)^p - 1 is its binomial series to delta^5 (the first omitted
// term is below 1e-18 for |delta| <= 2^-10; |delta| measured on the 2-D and
// 1-D workloads stays below 4e-6), in place of a log and an exp.  The log
// supersaturation follows as L = L0 + log1p(delta), the same series with
// log1p's coefficients in lane 3.  Lane k: rate of lane k (0 G1, 1 G2, 2 B),
// lane 3: L.
struct RateCarry {
    double c[5];     // the lane's series coefficients: C(p, k) (lanes 0-2, and up), (-1)^(k+1) / k (lane 3)
    double a, b;     // the lane's result is fma(a, P, b): a = b = G(d0) (rates), a = 1, b = L0 (lane 3)
    double d0, inv_d0;
    int ok;          // the stage-1 chain left a power-law evaluation at d0 > 0
};

__device__ __forceinline__ void rate_carry_init(RateCarry& rc, const Kin& K)
{
    const int lane = threadIdx.x & 31;
    const double p = lane == 0 ? K.g1 : (lane == 1 ? K.g2 : K.b);
    double ck = 1.0;
#pragma unroll
    for (int k = 1; k <= 5; ++k) {
        ck = ck * (p - (k - 1)) / k;   // C(p, k)
        rc.c[k - 1] = lane == 3 ? ((k & 1) ? 1.0 : -1.0) / k : ck;
    }
    rc.a = rc.b = rc.d0 = rc.inv_d0 = 0.0;
    rc.ok = 0;
}

// The scalar chain between the stages, for the chain warp of the fused
// kernel: the same arithmetic as finish_stage1_warp / finish_stage2_warp
// with prepare_step_warp and stage_coef_fast, arranged for latency: every
// lane reads the scalars it needs at once and keeps them in registers, the
// kinetics start at once, lane 0's bookkeeping is stores at the end, and the
// coefficients of the next stage come from registers.  tc: temperature and
// solubility at the step's end time.
// Keep a full evaluation (kinetics_warp_T with rec) in rc for the series.
__device__ __forceinline__ void rate_carry_keep(RateCarry& rc, const Kin& K, double G1, double G2, double B, double L,
                                                const double (&rec)[2])
{
    const int lane = threadIdx.x & 31;
    const double r = lane == 0 ? G1 : (lane == 1 ? G2 : B);
    rc.a = lane == 3 ? 1.0 : r;
    rc.b = lane == 3 ? L : r;
    rc.d0 = rec[0];
    rc.inv_d0 = rec[1];
    rc.ok = K.kind == PBE_KINETICS_POWER_LAW && K.growth_form != 2 && finite_nonzero_bits(rec[1]);
}

// The rates at (C, c*) by the series from the evaluation kept in rc (at the
// same time: the same c* and Arrhenius factor); false, with nothing set,
// where it does not apply (then the caller evaluates the kinetics).
__device__ __forceinline__ bool rates_by_series(const RateCarry& rc, double C, double cs, int ndim, double& G1,
                                                double& G2, double& B, double& L)
{
    if (!rc.ok) return false;
    const double dd = C - cs, delta = (dd - rc.d0) * rc.inv_d0;
    if (!(dd > 0.0 && fabs(delta) <= 0x1p-10)) return false;
    double P = fma(rc.c[4], delta, rc.c[3]);
    P = fma(P, delta, rc.c[2]);
    P = fma(P, delta, rc.c[1]);
    P = fma(P, delta, rc.c[0]);
    const double e = fma(rc.a, P * delta, rc.b);
    G1 = __shfl_sync(0xffffffffu, e, 0);
    G2 = ndim == 2 ? __shfl_sync(0xffffffffu, e, 1) : 0.0;
    B = __shfl_sync(0xffffffffu, e, 2);
    L = __shfl_sync(0xffffffffu, e, 3);
    return true;
}

// TAYLOR (with rc): keep this evaluation for the stage-2 chain's series.
template <bool POLY = true, bool TAYLOR = false>
__device__ __forceinline__ StageCoef fused_finish1(Scal* S, const Kin& K, const Geom& g, double V1, const KinT& tc,
                                                   RateCarry* rc = nullptr)
{
    const int lane = threadIdx.x & 31;
    const double C1 = S->C - K.kappa * (V1 - S->V0);
    const double dt = S->dt;
    const int clipped = S->clipped;
    double G1, G2, B, L, sG[3], rec[2];
    kinetics_warp_T<POLY>(K, C1, tc, G1, G2, B, &L, sG, TAYLOR ? rec : nullptr);
    if (TAYLOR) rate_carry_keep(*rc, K, G1, G2, B, L, rec);
    if (lane == 0) {
        S->C1 = C1;
        S->V1 = V1;
        S->M1 = 1.0;
        S->G1b = G1; S->G2b = G2; S->Bb = B; S->Lb = L; S->sGb1 = sG[0]; S->sGb2 = sG[1]; S->spb = sG[2];
        S->fbb = 0;
        if (!isfinite(V1) || !isfinite(G1) || !isfinite(G2) || !isfinite(B)) {
            S->status = PBE_ENONFINITE;
            S->done = 1;
        }
    }
    __syncwarp();
    StageCoef sc;
    sc.c1 = (G1 * g.inv_d1) * dt;
    sc.c2 = (G2 * g.inv_d2) * dt;
    sc.src = g.ndim == 1 ? (B * g.inv_d1) * dt : (B * (g.inv_d1 * g.inv_d2)) * dt;
    sc.moms = clipped != 0;
    return sc;
}

// TAYLOR (with rc): the rates by the series from the stage-1 chain's
// evaluation when it applies (RateCarry), else the full kinetics.
template <bool POLY = true, bool TAYLOR = false>
__device__ __forceinline__ StageCoef fused_finish2(Scal* S, const Kin& K, const Geom& g, const double* t_out,
                                                   double* rows, const double* mom, int nmom, int vidx,
                                                   const KinT& tc, const RateCarry* rc = nullptr)
{
    const int lane = threadIdx.x & 31;
    const double V2 = mom[vidx], M2 = mom[0];
    const double C = S->C - K.kappa * (V2 - S->V0);
    const double t = S->t_new, dt_done = S->dt;
    const int clipped = S->clipped, out_idx = S->out_idx, n_out = S->n_out;
    const long long steps = S->steps + 1, max_steps = S->max_steps;
    const bool finite = isfinite(V2) && isfinite(C);
    const int oi = (finite && clipped) ? out_idx + 1 : out_idx;
    const bool done = !finite || oi >= n_out || steps >= max_steps;
    __syncwarp();   // every lane has read S before lane 0 writes it
    double G1 = 0.0, G2 = 0.0, B = 0.0, dt = 0.0, t_new = t, L = 0.0, sG[3] = {0.0, 0.0, 0.0};
    int clip2 = 0;
    if (!done) {   // the next step: kinetics at (C, t), CFL step to the next output time
        const bool series = TAYLOR && rates_by_series(*rc, C, tc.cs, g.ndim, G1, G2, B, L);
        if (!series) kinetics_warp_T<POLY>(K, C, tc, G1, G2, B, &L, sG);
        clip2 = timestep_fast(K, g, G1, G2, t, t_out[oi], dt, t_new);
    }
    if (lane == 0) {
        S->t = t;
        S->C = C;
        S->V0 = V2;
        S->M0 = M2;
        S->last_dt = dt_done;
        S->steps = steps;
        if (!finite) {
            S->status = PBE_ENONFINITE;
            S->done = 1;
        } else {
            if (clipped) {
                if (rows) {
                    double* row = rows + (size_t)out_idx * (nmom + 2);
                    row[0] = t;
                    for (int k = 0; k < nmom; ++k) row[1 + k] = mom[k];
                    row[nmom + 1] = C;
                }
                S->out_idx = oi;
            }
            if (oi >= n_out) {
                S->done = 1;
            } else if (steps >= max_steps) {
                S->status = PBE_ETIMEOUT;
                S->done = 1;
            }
        }
        if (!done) {
            S->G1a = G1; S->G2a = G2; S->Ba = B; S->La = L; S->sGa1 = sG[0]; S->sGa2 = sG[1]; S->spa = sG[2];
            S->fba = 0;
            S->dt = dt; S->t_new = t_new; S->clipped = clip2;
            if (!isfinite(G1) || !isfinite(G2) || !isfinite(B) || !isfinite(dt)) {
                S->status = PBE_ENONFINITE;
                S->done = 1;
            }
        }
    }
    __syncwarp();
    StageCoef sc;
    sc.c1 = (G1 * g.inv_d1) * dt;
    sc.c2 = (G2 * g.inv_d2) * dt;
    sc.src = g.ndim == 1 ? (B * g.inv_d1) * dt : (B * (g.inv_d1 * g.inv_d2)) * dt;
    sc.moms = false;
    return sc;
}

}  // namespace pbe

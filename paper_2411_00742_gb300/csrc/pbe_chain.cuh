// The scalar chain between the two stages of a step, arranged for the
// latency of one warp (used by the persistent kernels): the solute balance
// of Eq. 4, the kinetics, the CFL step and the next stage's coefficients.
#pragma once

#include "pbe_tiles.cuh"

namespace pbe {

// The scalar chain between the stages, for the chain warp of the fused
// kernel: the same arithmetic as finish_stage1_warp / finish_stage2_warp
// with prepare_step_warp and stage_coef_fast, arranged for latency: every
// lane reads the scalars it needs at once and keeps them in registers, the
// kinetics start at once, lane 0's bookkeeping is stores at the end, and the
// coefficients of the next stage come from registers.  tc: temperature and
// solubility at the step's end time.
template <bool POLY = true>
__device__ __forceinline__ StageCoef fused_finish1(Scal* S, const Kin& K, const Geom& g, double V1, const KinT& tc)
{
    const int lane = threadIdx.x & 31;
    const double C1 = S->C - K.kappa * (V1 - S->V0);
    const double dt = S->dt;
    const int clipped = S->clipped;
    double G1, G2, B, L, sG[3];
    kinetics_warp_T<POLY>(K, C1, tc, G1, G2, B, &L, sG);
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

template <bool POLY = true>
__device__ __forceinline__ StageCoef fused_finish2(Scal* S, const Kin& K, const Geom& g, const double* t_out,
                                                   double* rows, const double* mom, int nmom, int vidx,
                                                   const KinT& tc)
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
        kinetics_warp_T<POLY>(K, C, tc, G1, G2, B, &L, sG);
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

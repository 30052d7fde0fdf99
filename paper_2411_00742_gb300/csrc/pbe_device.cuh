// Device-side building blocks shared by the plain and fused kernels:
// kinetic model, CFL step, limited face value, reductions and the scalar
// chain that closes the solute balance between stages.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pbe.h"
#include "pbe_math.cuh"

namespace pbe {

constexpr int kMaxMom = 10;  // moments per row: 4 (1-D) or 10 (2-D)

// Kinetic model and scheme constants, passed to kernels by value.
struct Kin {
    int kind, ndim;
    double kg1, g1, kg2, g2, kb, b;
    double cs0, cs1, cs2, T0, T1, t_cool, kappa, cfl;
    double lkg1, lkg2, lkb;   // natural logarithms of kg1, kg2, kb (-inf for 0)
    double inv_tcool;         // 1 / t_cool
};

struct Geom {
    int ndim;
    int N1, N2;      // cells along L1 and L2 (N2 = 1 in 1-D)
    double d1, d2;   // cell widths
    double inv_d1, inv_d2;
};

// Scalar state of one solve, resident in device memory between kernels.
struct Scal {
    double C, t, V0;            // state at the start of the current step
    double dt, t_new;           // current step
    double G1a, G2a, Ba;        // stage-1 kinetics (state at step start)
    double G1b, G2b, Bb;        // stage-2 kinetics (after stage 1)
    double C1;                  // concentration after stage 1
    double last_dt;             // length of the last completed step
    long long steps, max_steps;
    int clipped, out_idx, n_out, done, status;
    unsigned int counter;       // arrival counter of the last-block reductions
};

// S = C / c*(T), s = max(S - 1, 0); G_d = kg_d s^g_d, B = kb s^b (Sec. 2.1,
// Appendix A: growth only for S > 1).
__device__ __forceinline__ void kinetics(const Kin& K, double C, double t, double& G1, double& G2,
                                         double& B)
{
    if (K.kind == PBE_KINETICS_FIXED) {
        G1 = K.kg1;
        G2 = (K.ndim == 2) ? K.kg2 : 0.0;
        B = K.kb;
        return;
    }
    double frac = (t < K.t_cool) ? t / K.t_cool : 1.0;
    double T = K.T0 + (K.T1 - K.T0) * frac;
    double cs = K.cs0 + K.cs1 * T + K.cs2 * T * T;
    double s = C / cs - 1.0;
    if (!(s > 0.0)) {
        G1 = 0.0; G2 = 0.0; B = 0.0;
        return;
    }
    G1 = K.kg1 * pow(s, K.g1);
    G2 = (K.ndim == 2) ? K.kg2 * pow(s, K.g2) : 0.0;
    B = K.kb * pow(s, K.b);
}

// CFL step dt = cfl / (G1/dL1 + G2/dL2), clipped to end at t_next (SI Sec. S1.1).
__device__ __forceinline__ int timestep(const Kin& K, const Geom& g, double G1, double G2, double t,
                                        double t_next, double& dt, double& t_new)
{
    double rate = G1 / g.d1;
    if (g.ndim == 2) rate = rate + G2 / g.d2;
    double rem = t_next - t;
    if (rate > 0.0) {
        double dtc = K.cfl / rate;
        if (dtc < rem) {
            dt = dtc;
            t_new = t + dtc;
            return 0;
        }
    }
    dt = rem;
    t_new = t_next;
    return 1;
}

// Half the van Leer limited slope: phi(theta) (n_{i+1} - n_i) / 2 with
// theta = a / b, a = n_i - n_{i-1}, b = n_{i+1} - n_i (SI Sec. S1.1),
// i.e. a b / (a + b) when a and b have the same strict sign, else 0.
__device__ __forceinline__ double half_psi(double a, double b)
{
    double r = 0.0;
    if ((a > 0.0 && b > 0.0) || (a < 0.0 && b < 0.0)) r = a * (b / (a + b));
    return r;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum of NV values; the result is valid in thread 0.
// `sh` holds NT/32 * NV doubles.
template <int NT, int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[w * NV + k] = v[k];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = (lane < NT / 32) ? sh[lane * NV + k] : 0.0;
            v[k] = warp_sum(x);
        }
    }
    __syncthreads();
}

// Called by every thread after thread 0 stored this block's partials.
// Returns true in exactly one block: the last to arrive.
__device__ __forceinline__ bool last_block(unsigned int* counter, unsigned int nblocks, int* flag_sh)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int prev = atomicAdd(counter, 1u);
        *flag_sh = (prev == nblocks - 1u);
    }
    __syncthreads();
    bool last = *flag_sh != 0;
    if (last) __threadfence();
    return last;
}

// Sum the NV partials of all blocks in a fixed order (deterministic).
template <int NT, int NV>
__device__ __forceinline__ void reduce_partials(const double* part, int nblocks, double (&v)[NV],
                                                double* sh)
{
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0.0;
    for (int blk = threadIdx.x; blk < nblocks; blk += NT) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __ldcg(part + (size_t)blk * kMaxMom + k);
    }
    block_sum<NT, NV>(v, sh);
}

// Kinetics and step length of the next step from (C, t) (thread 0 only).
__device__ __forceinline__ void prepare_step(Scal* S, const Kin& K, const Geom& g, const double* t_out)
{
    double t_next = t_out[S->out_idx];
    double G1, G2, B, dt, t_new;
    kinetics(K, S->C, S->t, G1, G2, B);
    int clipped = timestep(K, g, G1, G2, S->t, t_next, dt, t_new);
    S->G1a = G1; S->G2a = G2; S->Ba = B;
    S->dt = dt; S->t_new = t_new; S->clipped = clipped;
    if (!isfinite(G1) || !isfinite(G2) || !isfinite(B) || !isfinite(dt)) {
        S->status = PBE_ENONFINITE;
        S->done = 1;
    }
}

// After stage 1: C1 = C - kappa (V(n1) - V(n)) (Eq. 4) and the stage-2
// kinetics at (C1, t + dt).
__device__ __forceinline__ void finish_stage1(Scal* S, const Kin& K, double V1)
{
    double C1 = S->C - K.kappa * (V1 - S->V0);
    double G1, G2, B;
    kinetics(K, C1, S->t_new, G1, G2, B);
    S->C1 = C1;
    S->G1b = G1; S->G2b = G2; S->Bb = B;
    if (!isfinite(V1) || !isfinite(G1) || !isfinite(G2) || !isfinite(B)) {
        S->status = PBE_ENONFINITE;
        S->done = 1;
    }
}

// After stage 2: close the step, emit an output row when the step landed on
// an output time, prepare the next step or finish.
__device__ __forceinline__ void finish_stage2(Scal* S, const Kin& K, const Geom& g, const double* t_out,
                                              double* rows, const double* mom, int nmom, int vidx)
{
    double V2 = mom[vidx];
    double C = S->C - K.kappa * (V2 - S->V0);
    S->t = S->t_new;
    S->C = C;
    S->V0 = V2;
    S->last_dt = S->dt;
    S->steps += 1;
    if (!isfinite(V2) || !isfinite(C)) {
        S->status = PBE_ENONFINITE;
        S->done = 1;
        return;
    }
    if (S->clipped) {
        if (rows) {  // rows == nullptr: a replica of the scalar chain that must not write
            double* row = rows + (size_t)S->out_idx * (nmom + 2);
            row[0] = S->t;
            for (int k = 0; k < nmom; ++k) row[1 + k] = mom[k];
            row[nmom + 1] = C;
        }
        S->out_idx += 1;
    }
    if (S->out_idx >= S->n_out) {
        S->done = 1;
    } else if (S->steps >= S->max_steps) {
        S->status = PBE_ETIMEOUT;
        S->done = 1;
    } else {
        prepare_step(S, K, g, t_out);
    }
}

// ---------------------------------------------------------------------------
// Warp-level scalar chain.  On GB300 a dependent FP64 operation takes ~65
// cycles and pow() several thousand, so the chain between stages is the
// latency that matters.  The same kinetics are computed with one logarithm
// pair and three exponentials spread over the lanes of one warp:
//   s^g = exp(g (ln(C - c*) - ln c*)),  kg s^g = exp(g ln s + ln kg),
// where C - c* is exact for S near 1.  Every lane of the calling warp must
// participate with identical arguments; all lanes return identical results.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void kinetics_warp(const Kin& K, double C, double t, double& G1, double& G2, double& B)
{
    const int lane = threadIdx.x & 31;
    if (K.kind == PBE_KINETICS_FIXED) {
        G1 = K.kg1;
        G2 = (K.ndim == 2) ? K.kg2 : 0.0;
        B = K.kb;
        return;
    }
    const double frac = (t < K.t_cool) ? t * K.inv_tcool : 1.0;
    const double T = K.T0 + (K.T1 - K.T0) * frac;
    const double cs = K.cs0 + K.cs1 * T + K.cs2 * T * T;
    const double d = C - cs;
    if (!(d > 0.0)) {   // S <= 1: no growth, no nucleation
        G1 = 0.0; G2 = 0.0; B = 0.0;
        return;
    }
    const double lx = pbe_log(lane == 0 ? d : cs);
    const double L = __shfl_sync(0xffffffffu, lx, 0) - __shfl_sync(0xffffffffu, lx, 1);
    const double p = lane == 0 ? K.g1 : (lane == 1 ? K.g2 : K.b);
    const double q = lane == 0 ? K.lkg1 : (lane == 1 ? K.lkg2 : K.lkb);
    const double e = pbe_exp(fma(p, L, q));
    G1 = __shfl_sync(0xffffffffu, e, 0);
    G2 = (K.ndim == 2) ? __shfl_sync(0xffffffffu, e, 1) : 0.0;
    B = __shfl_sync(0xffffffffu, e, 2);
}

__device__ __forceinline__ int timestep_fast(const Kin& K, const Geom& g, double G1, double G2, double t,
                                             double t_next, double& dt, double& t_new)
{
    double rate = G1 * g.inv_d1;
    if (g.ndim == 2) rate = fma(G2, g.inv_d2, rate);
    const double rem = t_next - t;
    if (rate > 0.0) {
        const double dtc = K.cfl / rate;
        if (dtc < rem) {
            dt = dtc;
            t_new = t + dtc;
            return 0;
        }
    }
    dt = rem;
    t_new = t_next;
    return 1;
}

// Warp versions of prepare_step / finish_stage1 / finish_stage2: called by all
// lanes of one warp on the same Scal (shared or global); lane 0 writes.
__device__ __forceinline__ void prepare_step_warp(Scal* S, const Kin& K, const Geom& g, const double* t_out)
{
    const int lane = threadIdx.x & 31;
    const double t_next = t_out[S->out_idx];
    const double C = S->C, t = S->t;
    double G1, G2, B, dt, t_new;
    kinetics_warp(K, C, t, G1, G2, B);
    const int clipped = timestep_fast(K, g, G1, G2, t, t_next, dt, t_new);
    __syncwarp();
    if (lane == 0) {
        S->G1a = G1; S->G2a = G2; S->Ba = B;
        S->dt = dt; S->t_new = t_new; S->clipped = clipped;
        if (!isfinite(G1) || !isfinite(G2) || !isfinite(B) || !isfinite(dt)) {
            S->status = PBE_ENONFINITE;
            S->done = 1;
        }
    }
    __syncwarp();
}

__device__ __forceinline__ void finish_stage1_warp(Scal* S, const Kin& K, double V1)
{
    const int lane = threadIdx.x & 31;
    const double C1 = S->C - K.kappa * (V1 - S->V0);
    double G1, G2, B;
    kinetics_warp(K, C1, S->t_new, G1, G2, B);
    __syncwarp();
    if (lane == 0) {
        S->C1 = C1;
        S->G1b = G1; S->G2b = G2; S->Bb = B;
        if (!isfinite(V1) || !isfinite(G1) || !isfinite(G2) || !isfinite(B)) {
            S->status = PBE_ENONFINITE;
            S->done = 1;
        }
    }
    __syncwarp();
}

__device__ __forceinline__ void finish_stage2_warp(Scal* S, const Kin& K, const Geom& g, const double* t_out,
                                                   double* rows, const double* mom, int nmom, int vidx)
{
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        const double V2 = mom[vidx];
        const double C = S->C - K.kappa * (V2 - S->V0);
        S->t = S->t_new;
        S->C = C;
        S->V0 = V2;
        S->last_dt = S->dt;
        S->steps += 1;
        if (!isfinite(V2) || !isfinite(C)) {
            S->status = PBE_ENONFINITE;
            S->done = 1;
        } else {
            if (S->clipped) {
                if (rows) {
                    double* row = rows + (size_t)S->out_idx * (nmom + 2);
                    row[0] = S->t;
                    for (int k = 0; k < nmom; ++k) row[1 + k] = mom[k];
                    row[nmom + 1] = C;
                }
                S->out_idx += 1;
            }
            if (S->out_idx >= S->n_out) {
                S->done = 1;
            } else if (S->steps >= S->max_steps) {
                S->status = PBE_ETIMEOUT;
                S->done = 1;
            }
        }
    }
    __syncwarp();
    if (!S->done) prepare_step_warp(S, K, g, t_out);
}

}  // namespace pbe

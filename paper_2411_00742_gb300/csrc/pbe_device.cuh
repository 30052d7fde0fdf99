// Device-side building blocks shared by the plain and fused kernels:
// kinetic model, CFL step, limited face value, reductions and the scalar
// chain that closes the solute balance between stages.
#pragma once

#include <cuda_bf16.h>
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
    int scheme;               // PBE_SCHEME_*
    int growth_form, solubility_form;
    double ea1, ea2;          // Arrhenius activation temperatures (growth_form 1)
    const __nv_bfloat16* mW;  // learned closure: W1[64][3], W2[64][64], W3[3][64] (bf16, device)
    const float* mB;          // and b1[64], b2[64], b3[3] (fp32, device)
    const double* poly;       // growth_form 2 (Eq. 6): a[m * npoly + k - 1], k = 1..npoly, m < ndim (device)
    int npoly;
    int mbox;                 // learned closure: 1 if its inputs have a training box [mlo, mhi]
    double mlo[3], mhi[3];
};

constexpr int kMlpH = 64;
constexpr int kMlpNW = kMlpH * 3 + kMlpH + kMlpH * kMlpH + kMlpH + 3 * kMlpH + 3;  // flat weight count

// The integer w as a double, exactly, for 0 <= w < 2^52: w in the low
// mantissa bits of 2^52, minus 2^52 (one FP64 addition, no conversion).
__device__ __forceinline__ double exact_int_double(long long w)
{
    return __longlong_as_double(0x4330000000000000LL | w) - 4503599627370496.0;
}

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
    double M0;                  // mu0 of the state at the start of the step
    double V1, M1;              // volume moment and mu0 after stage 1
    double last_dt;             // length of the last completed step
    long long steps, max_steps;
    int clipped, out_idx, n_out, done, status;
    int row_first;              // first row a fused solve emitted (its moments are summed afterwards)
    unsigned int counter;       // arrival counter of the last-block reductions
    double La, Lb;              // ln s of the stage-1 and stage-2 power-law kinetics (warp chains;
                                // 0 when S <= 1), kept for the adjoint
    double sGa1, sGa2, sGb1, sGb2;  // s dG_m/ds of the polynomial growth law (Eq. 6) at both stages
    double spa, spb;                // s = S - 1 at both stages (polynomial growth law)
    int fba, fbb;                   // learned closure: 1 if the stage took the power-law fallback
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
    double cs = K.solubility_form == 1 ? K.cs0 * exp(K.cs1 * T) : K.cs0 + K.cs1 * T + K.cs2 * T * T;
    double s = C / cs - 1.0;
    if (!(s > 0.0)) {
        G1 = 0.0; G2 = 0.0; B = 0.0;
        return;
    }
    const double a1 = K.growth_form == 1 ? exp(-K.ea1 / (T + 273.15)) : 1.0;
    const double a2 = K.growth_form == 1 ? exp(-K.ea2 / (T + 273.15)) : 1.0;
    G1 = K.kg1 * a1 * pow(s, K.g1);
    G2 = (K.ndim == 2) ? K.kg2 * a2 * pow(s, K.g2) : 0.0;
    B = K.kb * pow(s, K.b);
}

// CFL step dt = cfl / (G1/dL1 + G2/dL2), clipped to end at t_next (SI Sec. S1.1).
__device__ __forceinline__ int timestep(const Kin& K, const Geom& g, double G1, double G2, double t,
                                        double t_next, double& dt, double& t_new)
{
    double rate = G1 / g.d1;
    if (g.ndim == 2) {
        const double r2 = G2 / g.d2;
        rate = K.scheme == PBE_SCHEME_PAPER ? (r2 > rate ? r2 : rate) : rate + r2;
    }
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

// Differences below this magnitude count as flat for the limiter's
// derivative (their ratio is decided by rounding of underflowing tails).
constexpr double kPsiFlat = 0x1p-959;

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
// Temperature and solubility at time t (they depend on t only, so a caller
// that evaluates the kinetics twice at one time can compute them once).
struct KinT {
    double T, cs;
};

__device__ __forceinline__ KinT kin_temperature(const Kin& K, double t)
{
    const double frac = (t < K.t_cool) ? t * K.inv_tcool : 1.0;
    const double T = K.T0 + (K.T1 - K.T0) * frac;
    const double cs = K.solubility_form == 1 ? K.cs0 * pbe_exp_tab(K.cs1 * T) : K.cs0 + K.cs1 * T + K.cs2 * T * T;
    return KinT{T, cs};
}

// The polynomial growth law of Eq. 6, G_m = sum_{k=1..K} a_mk s^k, and
// s dG_m/ds = sum_k k a_mk s^k, for both directions, on one warp: lane l takes
// the terms k0 .. k0 + c - 1 (c = ceil(K / 32), k0 = l c + 1) by Horner's rule
// in s, scaled by s^k0 = exp(k0 ln s); a butterfly sums the lanes (the same
// result in every lane).
__device__ __forceinline__ void poly_growth_warp(const Kin& K, double s, double L, double& G1, double& G2,
                                                 double& sG1, double& sG2)
{
    const int lane = threadIdx.x & 31, n = K.npoly;
    const int c = (n + 31) >> 5, k0 = lane * c + 1;
    double g[2] = {0.0, 0.0}, h[2] = {0.0, 0.0};
    if (k0 <= n) {
        const int k1 = min(n, k0 + c - 1);
        const double sk0 = k0 == 1 ? s : pbe_exp_tab((double)k0 * L);
        for (int m = 0; m < K.ndim; ++m) {
            const double* a = K.poly + (size_t)m * n;
            double pg = 0.0, ph = 0.0;
            for (int k = k1; k >= k0; --k) {
                const double ak = __ldg(a + k - 1);
                pg = fma(pg, s, ak);
                ph = fma(ph, s, (double)k * ak);
            }
            g[m] = pg * sk0;
            h[m] = ph * sk0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        g[0] += __shfl_xor_sync(0xffffffffu, g[0], o);
        g[1] += __shfl_xor_sync(0xffffffffu, g[1], o);
        h[0] += __shfl_xor_sync(0xffffffffu, h[0], o);
        h[1] += __shfl_xor_sync(0xffffffffu, h[1], o);
    }
    G1 = g[0];
    G2 = K.ndim == 2 ? g[1] : 0.0;
    sG1 = h[0];
    sG2 = K.ndim == 2 ? h[1] : 0.0;
}

// Lout (optional) receives ln s (0 for fixed kinetics or S <= 1); sGout
// (optional, 3 values) s dG_1/ds, s dG_2/ds and s of the polynomial growth
// law (0 otherwise).  POLY false: a caller that never sees the polynomial law
// (the fused solve kernel; its register budget sets its occupancy).
// rec (optional, 2 values): d = C - c* and 1/d (0, 0 when S <= 1 or the
// rates are fixed), 1/d from lane 3 of the exp, which runs in every lane.
template <bool POLY = true>
__device__ __forceinline__ void kinetics_warp_T(const Kin& K, double C, const KinT& tc, double& G1, double& G2,
                                                double& B, double* Lout = nullptr, double* sGout = nullptr,
                                                double* rec = nullptr)
{
    const int lane = threadIdx.x & 31;
    if (Lout) *Lout = 0.0;
    if (rec) { rec[0] = 0.0; rec[1] = 0.0; }
    if (sGout) { sGout[0] = 0.0; sGout[1] = 0.0; sGout[2] = 0.0; }
    if (K.kind == PBE_KINETICS_FIXED) {
        G1 = K.kg1;
        G2 = (K.ndim == 2) ? K.kg2 : 0.0;
        B = K.kb;
        return;
    }
    const double T = tc.T, cs = tc.cs;
    const double d = C - cs;
    if (!(d > 0.0)) {   // S <= 1: no growth, no nucleation
        G1 = 0.0; G2 = 0.0; B = 0.0;
        return;
    }
    const double lx = pbe_log_tab(lane == 0 ? d : cs);
    const double ld = __shfl_sync(0xffffffffu, lx, 0);
    const double L = ld - __shfl_sync(0xffffffffu, lx, 1);
    if (Lout) *Lout = L;
    const double p = lane == 0 ? K.g1 : (lane == 1 ? K.g2 : K.b);
    double q = lane == 0 ? K.lkg1 : (lane == 1 ? K.lkg2 : K.lkb);
    if (K.growth_form == 1 && lane < 2) q -= (lane == 0 ? K.ea1 : K.ea2) / (T + 273.15);   // Arrhenius factor
    double arg = fma(p, L, q);
    if (rec && lane == 3) arg = -ld;
    const double e = pbe_exp_tab(arg);
    if (rec) { rec[0] = d; rec[1] = __shfl_sync(0xffffffffu, e, 3); }
    G1 = __shfl_sync(0xffffffffu, e, 0);
    G2 = (K.ndim == 2) ? __shfl_sync(0xffffffffu, e, 1) : 0.0;
    B = __shfl_sync(0xffffffffu, e, 2);
    if (POLY && K.growth_form == 2) {   // Eq. 6 in place of the power law; nucleation keeps its law
        double sG1, sG2;
        const double sp = d * __drcp_rn(cs);
        poly_growth_warp(K, sp, L, G1, G2, sG1, sG2);
        if (sGout) { sGout[0] = sG1; sGout[1] = sG2; sGout[2] = sp; }
    }
}

template <bool POLY = true>
__device__ __forceinline__ void kinetics_warp(const Kin& K, double C, double t, double& G1, double& G2, double& B,
                                              double* Lout = nullptr, double* sGout = nullptr)
{
    if (K.kind == PBE_KINETICS_FIXED) {
        kinetics_warp_T<POLY>(K, C, KinT{0.0, 0.0}, G1, G2, B, Lout, sGout);
        return;
    }
    kinetics_warp_T<POLY>(K, C, kin_temperature(K, t), G1, G2, B, Lout, sGout);
}

// ---------------------------------------------------------------------------
// Learned closure (a perceptron replaces the rate expressions: the empirical
// hybrid model of Sec. 4.2): 3 -> 64 -> 64 -> 3 with SiLU hidden units, bf16
// weights, fp32 arithmetic and accumulation, one warp (two hidden units per
// lane).  Inputs x0 = 4 (S - 1), x1 = (T - 25)/10, x2 = 1e-6 V/mu0; outputs
// ln G1 = o0 + ln 0.01, ln G2 = o1 + ln 0.005, ln B = o2 + ln 1e5.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }

__device__ __forceinline__ void mlp_forward_warp(const Kin& K, const float x[3], float o[3])
{
    const int lane = threadIdx.x & 31;
    const __nv_bfloat16* W1 = K.mW;
    const __nv_bfloat16* W2 = W1 + kMlpH * 3;
    const __nv_bfloat16* W3 = W2 + kMlpH * kMlpH;
    const float* b1 = K.mB;
    const float* b2 = b1 + kMlpH;
    const float* b3 = b2 + kMlpH;
    float a1[2], z2[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int h = lane + 32 * u;
        float z = b1[h];
        z = fmaf(__bfloat162float(W1[h * 3]), x[0], z);
        z = fmaf(__bfloat162float(W1[h * 3 + 1]), x[1], z);
        z = fmaf(__bfloat162float(W1[h * 3 + 2]), x[2], z);
        a1[u] = silu_f(z);
        z2[u] = b2[h];
    }
    for (int j = 0; j < 32; ++j) {
        const float aj0 = __shfl_sync(0xffffffffu, a1[0], j), aj1 = __shfl_sync(0xffffffffu, a1[1], j);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int h = lane + 32 * u;
            z2[u] = fmaf(__bfloat162float(W2[h * kMlpH + j]), aj0, z2[u]);
            z2[u] = fmaf(__bfloat162float(W2[h * kMlpH + j + 32]), aj1, z2[u]);
        }
    }
    const float a20 = silu_f(z2[0]), a21 = silu_f(z2[1]);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        float v = __bfloat162float(W3[m * kMlpH + lane]) * a20 + __bfloat162float(W3[m * kMlpH + lane + 32]) * a21;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        o[m] = v + b3[m];
    }
}

// closure inputs in FP64 at (C, t, ratio); returns false when S <= 1
__device__ __forceinline__ bool mlp_inputs_d(const Kin& K, double C, double t, double ratio, double x[3])
{
    const double frac = (t < K.t_cool) ? t * K.inv_tcool : 1.0;
    const double T = K.T0 + (K.T1 - K.T0) * frac;
    const double cs = K.cs0 + K.cs1 * T + K.cs2 * T * T;
    const double s = C / cs - 1.0;
    if (!(s > 0.0)) return false;
    x[0] = 4.0 * s;
    x[1] = (T - 25.0) / 10.0;
    x[2] = 1e-6 * ratio;
    return true;
}

// closure inputs at (C, t, ratio); returns false when S <= 1
__device__ __forceinline__ bool mlp_inputs(const Kin& K, double C, double t, double ratio, float x[3])
{
    const double frac = (t < K.t_cool) ? t * K.inv_tcool : 1.0;
    const double T = K.T0 + (K.T1 - K.T0) * frac;
    const double cs = K.cs0 + K.cs1 * T + K.cs2 * T * T;
    const double s = C / cs - 1.0;
    if (!(s > 0.0)) return false;
    x[0] = (float)(4.0 * s);
    x[1] = (float)((T - 25.0) / 10.0);
    x[2] = (float)(1e-6 * ratio);
    return true;
}

constexpr double kLnG1 = -4.605170185988091;   // ln 0.01
constexpr double kLnG2 = -5.298317366548036;   // ln 0.005
constexpr double kLnB = 11.512925464970229;    // ln 1e5

// kinetics with the moment ratio V/mu0 of the state (used by the closure);
// pre: temperature and solubility at t when the caller has them
// The learned closure's plain-kinetics fallback: the power law of the
// kinetic parameters replaces the network when an input (FP64) leaves the
// training box (if one is set) or a rate is not finite; fbout (optional)
// receives 1 when it did.
__device__ __forceinline__ void kinetics_warp_r(const Kin& K, double C, double t, double ratio, double& G1,
                                                double& G2, double& B, const KinT* pre = nullptr,
                                                double* Lout = nullptr, double* sGout = nullptr,
                                                int* fbout = nullptr)
{
    if (fbout) *fbout = 0;
    if (K.kind != PBE_KINETICS_MLP) {
        if (pre) kinetics_warp_T(K, C, *pre, G1, G2, B, Lout, sGout);
        else kinetics_warp(K, C, t, G1, G2, B, Lout, sGout);
        return;
    }
    if (Lout) *Lout = 0.0;
    if (sGout) { sGout[0] = 0.0; sGout[1] = 0.0; sGout[2] = 0.0; }
    double xd[3];
    if (!mlp_inputs_d(K, C, t, ratio, xd)) {
        G1 = 0.0; G2 = 0.0; B = 0.0;
        return;
    }
    bool fb = false;
    if (K.mbox)
        for (int k = 0; k < 3; ++k) fb = fb || !(xd[k] >= K.mlo[k] && xd[k] <= K.mhi[k]);
    if (!fb) {
        const float x[3] = {(float)xd[0], (float)xd[1], (float)xd[2]};
        float o[3];
        mlp_forward_warp(K, x, o);
        G1 = pbe_exp_tab((double)o[0] + kLnG1);
        G2 = (K.ndim == 2) ? pbe_exp_tab((double)o[1] + kLnG2) : 0.0;
        B = pbe_exp_tab((double)o[2] + kLnB);
        fb = !(isfinite(G1) && isfinite(G2) && isfinite(B));
    }
    if (fb) {   // the power law (kind != FIXED, growth_form 0 for the closure)
        if (pre) kinetics_warp_T(K, C, *pre, G1, G2, B, Lout, sGout);
        else kinetics_warp(K, C, t, G1, G2, B, Lout, sGout);
        if (fbout) *fbout = 1;
    }
}

// a / b for b > 0 (finite) by Newton-Raphson: from the hardware reciprocal
// approximation y0 (relative error e = 1 - b y0 below 2^-20), the first-order
// refinements of the reciprocal, y1 = y0 + y0 e, and of the quotient,
// q1 = a y0 + (a y0) e, side by side (relative error ~e^2), then one residual
// correction q1 + y1 (a - b q1) (error ~e^4, below the rounding), which leaves
// the result within an ulp of the rounded quotient: four dependent FP64
// operations after the approximation.
__device__ __forceinline__ double div_newton(double a, double b)
{
    double y0;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(b));
    const double e = fma(-b, y0, 1.0), q0 = a * y0;
    const double y1 = fma(y0, e, y0), q1 = fma(q0, e, q0);
    return fma(y1, fma(-b, q1, a), q1);
}

__device__ __forceinline__ int timestep_fast(const Kin& K, const Geom& g, double G1, double G2, double t,
                                             double t_next, double& dt, double& t_new)
{
    double rate = G1 * g.inv_d1;
    if (g.ndim == 2) {
        if (K.scheme == PBE_SCHEME_PAPER) {
            const double r2 = G2 * g.inv_d2;
            rate = r2 > rate ? r2 : rate;
        } else {
            rate = fma(G2, g.inv_d2, rate);
        }
    }
    const double rem = t_next - t;
    if (rate > 0.0) {
        // (rates beyond ~1e307, whose reciprocal is subnormal, give dtc = 0 or
        // NaN here instead of a step of ~1e-300 s: either way no progress)
        const double dtc = div_newton(K.cfl, rate);
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
__device__ __forceinline__ void prepare_step_warp(Scal* S, const Kin& K, const Geom& g, const double* t_out,
                                                  const KinT* pre = nullptr)
{
    const int lane = threadIdx.x & 31;
    const double t_next = t_out[S->out_idx];
    const double C = S->C, t = S->t;
    double G1, G2, B, dt, t_new, L, sG[3];
    int fb;
    kinetics_warp_r(K, C, t, K.kind == PBE_KINETICS_MLP ? S->V0 / S->M0 : 0.0, G1, G2, B, pre, &L, sG, &fb);
    const int clipped = timestep_fast(K, g, G1, G2, t, t_next, dt, t_new);
    __syncwarp();
    if (lane == 0) {
        S->G1a = G1; S->G2a = G2; S->Ba = B; S->La = L; S->sGa1 = sG[0]; S->sGa2 = sG[1]; S->spa = sG[2];
        S->fba = fb;
        S->dt = dt; S->t_new = t_new; S->clipped = clipped;
        if (!isfinite(G1) || !isfinite(G2) || !isfinite(B) || !isfinite(dt)) {
            S->status = PBE_ENONFINITE;
            S->done = 1;
        }
    }
    __syncwarp();
}

// pre (optional): temperature and solubility at S->t_new
__device__ __forceinline__ void finish_stage1_warp(Scal* S, const Kin& K, double V1, double M1 = 1.0,
                                                   const KinT* pre = nullptr)
{
    const int lane = threadIdx.x & 31;
    const double C1 = S->C - K.kappa * (V1 - S->V0);
    double G1, G2, B, L, sG[3];
    int fb;
    kinetics_warp_r(K, C1, S->t_new, K.kind == PBE_KINETICS_MLP ? V1 / M1 : 0.0, G1, G2, B, pre, &L, sG, &fb);
    __syncwarp();
    if (lane == 0) {
        S->C1 = C1;
        S->V1 = V1;
        S->M1 = M1;
        S->G1b = G1; S->G2b = G2; S->Bb = B; S->Lb = L; S->sGb1 = sG[0]; S->sGb2 = sG[1]; S->spb = sG[2];
        S->fbb = fb;
        if (!isfinite(V1) || !isfinite(G1) || !isfinite(G2) || !isfinite(B)) {
            S->status = PBE_ENONFINITE;
            S->done = 1;
        }
    }
    __syncwarp();
}

// pre (optional): temperature and solubility at S->t_new (the time the next
// step starts from)
__device__ __forceinline__ void finish_stage2_warp(Scal* S, const Kin& K, const Geom& g, const double* t_out,
                                                   double* rows, const double* mom, int nmom, int vidx,
                                                   const KinT* pre = nullptr)
{
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        const double V2 = mom[vidx];
        const double C = S->C - K.kappa * (V2 - S->V0);
        S->t = S->t_new;
        S->C = C;
        S->V0 = V2;
        S->M0 = mom[0];
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
    if (!S->done) prepare_step_warp(S, K, g, t_out, pre);
}

}  // namespace pbe

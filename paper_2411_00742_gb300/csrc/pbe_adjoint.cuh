// Device building blocks of the discrete adjoint (reverse mode through the
// SSP-RK2 step, Sec. 4.1 gradients), shared by the per-stage adjoint kernels
// and the persistent one: moment-weight polynomials of the pending terms,
// the derivative data of one limited face, and the backward of the kinetics
// and of the learned closure.
#pragma once

#include "pbe_tiles.cuh"

namespace pbe {

// moment weight W_k at cell (i, j): x1^p x2^q dA (1-D: x^k dL)
template <int NDIM>
__device__ __forceinline__ double poly_weights(const double* pc, double x1, double x2, double dA)
{
    if (NDIM == 1) return (pc[0] + x1 * (pc[1] + x1 * (pc[2] + x1 * pc[3]))) * dA;
    // order mu00, mu10, mu01, mu20, mu11, mu02, mu30, mu21, mu12, mu03
    const double q0 = pc[0] + x2 * (pc[2] + x2 * (pc[5] + x2 * pc[9]));
    const double q1 = pc[1] + x2 * (pc[4] + x2 * pc[8]);
    const double q2 = pc[3] + x2 * pc[7];
    const double q3 = pc[6];
    return (q0 + x1 * (q1 + x1 * (q2 + x1 * q3))) * dA;
}

// derivative data of one face: contributions to the cells f-2, f-1, f and h
struct FaceAdj {
    double cm2, cm1, c0, hmu;
};

__device__ __forceinline__ FaceAdj face_adj(double nm2, double up, double dn, double lamL, double lamR, double invd)
{
    const double a = up - nm2, b = dn - up;
    double pa = 0.0, pb = 0.0, half = 0.0;
    if ((a > 0.0 && b > 0.0) || (a < 0.0 && b < 0.0)) {
        if (fabs(a) >= kPsiFlat && fabs(b) >= kPsiFlat) {
            // one division per face; |a + b| >= 2^-958, so 1 / (a + b) is finite
            const double rs = 1.0 / (a + b);
            const double qa = b * rs, qb = a * rs;
            half = a * qa;
            pa = 2.0 * qa * qa;
            pb = 2.0 * qb * qb;
        } else {
            // differences below 2^-959 count as flat for the derivative (their
            // ratio is decided by rounding of underflowing tails); the
            // reciprocal of their sum may overflow, the quotient does not
            half = a * (b / (a + b));
        }
    }
    const double mu = (lamR - lamL) * invd;
    FaceAdj r;
    r.cm2 = -0.5 * pa * mu;
    r.cm1 = (1.0 + 0.5 * (pa - pb)) * mu;
    r.c0 = 0.5 * pb * mu;
    r.hmu = (up + half) * mu;
    return r;
}

// Derivative data of the face with upwind-upwind, upwind and downwind cells
// (nm2, up, dn) for the fast forward: h = up + a q, a = up - nm2,
// b = dn - up, q = b/(a+b) (reciprocal approximation refined twice) when a
// and b have the same strict sign and both magnitudes reach 2^-959 (the
// forward's flat threshold), else h = up.  Returns mu times dh/d(nm2, up, dn)
// and h mu, mu = (lamR - lamL) / dL.
__device__ __forceinline__ FaceAdj face_adj_fast(double nm2, double up, double dn, double lamL, double lamR,
                                                 double invd)
{
    const double a = up - nm2, b = dn - up;
    const int ha = __double2hiint(a), hb = __double2hiint(b);
    const bool same = ((ha ^ hb) >= 0) && ((ha & 0x7ff00000) >= 0x04000000) && ((hb & 0x7ff00000) >= 0x04000000);
    const double mu = (lamR - lamL) * invd;
    FaceAdj r;
    if (same) {
        const double s = a + b;
        double rc;
        asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(rc) : "d"(s));
        rc = fma(rc, fma(-s, rc, 1.0), rc);
        rc = fma(rc, fma(-s, rc, 1.0), rc);
        const double q = b * rc, qm = q * mu, p = 1.0 - q;
        r.cm2 = -q * qm;
        r.cm1 = 2.0 * qm;
        r.c0 = (p * mu) * p;
        r.hmu = fma(a, q, up) * mu;
    } else {
        r.cm2 = 0.0;
        r.cm1 = mu;
        r.c0 = 0.0;
        r.hmu = up * mu;
    }
    return r;
}

// Backward of the rates at (C, t) given lG* = dL/dG* and the forward's rates
// and L = ln s (power law: dG/dkg = s^g = G/kg, dG/dg = G L, dG/ds = g G/s;
// no exponential or logarithm unless a prefactor is 0).  Adds to lth, *lC, *lt.
// s^g when the prefactor is 0 (the rate itself is then 0 and cannot give it);
// a call of its own so that the exponential is not evaluated speculatively
static __device__ __noinline__ double pow_from_log(double g, double L) { return pbe_exp_tab(g * L); }

// sG1, sG2: s dG_m/ds of the polynomial growth law (Eq. 6), recorded by the
// forward chain; that law's coefficient gradients are accumulated separately
// (poly_grad_accumulate), its dL/dkg and dL/dg entries stay 0.
__device__ __forceinline__ void kin_backward(const Kin& K, const double* ik, double C, double t, double G1, double G2,
                                             double B, double L, double sG1, double sG2, double lG1, double lG2,
                                             double lB, double* lC, double* lt, double* lth)
{
    if (K.kind == PBE_KINETICS_FIXED) {
        lth[0] += lG1;
        if (K.ndim == 2) lth[2] += lG2;
        lth[4] += lB;
        return;
    }
    // temperature and the polynomial solubility (the adjoint's only form), as kin_temperature
    const double frac = (t < K.t_cool) ? t * K.inv_tcool : 1.0;
    const double T = K.T0 + (K.T1 - K.T0) * frac;
    const double cs = K.cs0 + K.cs1 * T + K.cs2 * T * T;
    const double d = C - cs;
    if (!(d > 0.0)) return;   // S <= 1: the forward's rates were 0 whatever the parameters
    const double dTdt = (t < K.t_cool) ? (K.T1 - K.T0) * K.inv_tcool : 0.0;
    const double dcs = K.cs1 + 2.0 * K.cs2 * T;
    const double rd = __drcp_rn(d), rcs = __drcp_rn(cs);
    if (K.growth_form == 2) {
        double sb;
        if (K.kb > 0.0) sb = B * ik[2];
        else sb = pow_from_log(K.b, L);
        lth[4] += lB * sb;
        lth[5] += lB * B * L;
        const double q = (lG1 * sG1 + lG2 * sG2 + lB * K.b * B) * rd;
        *lC += q;
        *lt -= q * (C * rcs) * dcs * dTdt;
        return;
    }
    double s1, sb;
    if (K.kg1 > 0.0) s1 = G1 * ik[0];
    else s1 = pow_from_log(K.g1, L);
    if (K.kb > 0.0) sb = B * ik[2];
    else sb = pow_from_log(K.b, L);
    double num = lG1 * K.g1 * G1 + lB * K.b * B;   // s dL/ds
    lth[0] += lG1 * s1;
    lth[1] += lG1 * G1 * L;
    lth[4] += lB * sb;
    lth[5] += lB * B * L;
    if (K.ndim == 2) {
        double s2;
        if (K.kg2 > 0.0) s2 = G2 * ik[1];
        else s2 = pow_from_log(K.g2, L);
        lth[2] += lG2 * s2;
        lth[3] += lG2 * G2 * L;
        num += lG2 * K.g2 * G2;
    }
    // s = (C - c*)/c*: dL/dC = (dL/ds) / c* = num / (C - c*); dL/dt through c*(T(t))
    const double q = num * rd;
    *lC += q;
    *lt -= q * (C * rcs) * dcs * dTdt;
}

// ---------------------------------------------------------------------------
// scalar adjoint chain (one thread)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void kinetics_adjoint(const Kin& K, double C, double t, double lG1, double lG2, double lB, double* lC,
                                 double* lt, double* lth)
{
    if (K.kind == PBE_KINETICS_FIXED) {
        lth[0] += lG1;
        if (K.ndim == 2) lth[2] += lG2;
        lth[4] += lB;
        return;
    }
    const double frac = (t < K.t_cool) ? t / K.t_cool : 1.0;
    const double T = K.T0 + (K.T1 - K.T0) * frac;
    const double dTdt = (t < K.t_cool) ? (K.T1 - K.T0) / K.t_cool : 0.0;
    const double cs = K.cs0 + K.cs1 * T + K.cs2 * T * T;
    const double dcs = K.cs1 + 2.0 * K.cs2 * T;
    const double s = C / cs - 1.0;
    if (!(s > 0.0)) return;
    const double ls = log(s);
    const double s1 = exp(K.g1 * ls), sb = exp(K.b * ls);
    const double G1 = K.kg1 * s1, B = K.kb * sb;
    double lsum = lG1 * K.g1 * G1 / s + lB * K.b * B / s;
    lth[0] += lG1 * s1;
    lth[1] += lG1 * G1 * ls;
    lth[4] += lB * sb;
    lth[5] += lB * B * ls;
    if (K.ndim == 2) {
        const double s2 = exp(K.g2 * ls), G2 = K.kg2 * s2;
        lth[2] += lG2 * s2;
        lth[3] += lG2 * G2 * ls;
        lsum += lG2 * K.g2 * G2 / s;
    }
    *lC += lsum / cs;
    *lt += lsum * (-C * dcs / (cs * cs)) * dTdt;
}

// __syncthreads for the 64-thread blocks of the per-stage adjoint
struct BlockSync64 {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Backward of the learned closure for one evaluation, on 64 threads (one per
// hidden unit): recomputes the activations from the inputs x, takes the
// output adjoints lo = dL/d(o), accumulates dL/dweights into dW (fp64, flat
// layout W1, b1, W2, b2, W3, b3; nothing when dW is null) and returns dL/dx
// in lx (thread 0).  `sync` synchronizes the 64 threads.
template <class Sync>
__device__ __forceinline__ void mlp_backward_block64(const Kin& K, const float x[3], const double lo[3], double* dW,
                                                     float* sm, float lx[3], Sync sync)
{
    const int h = threadIdx.x;
    const __nv_bfloat16* W1 = K.mW;
    const __nv_bfloat16* W2 = W1 + kMlpH * 3;
    const __nv_bfloat16* W3 = W2 + kMlpH * kMlpH;
    const float* b1 = K.mB;
    const float* b2 = b1 + kMlpH;
    double* dW1 = dW;
    double* db1 = dW1 + kMlpH * 3;
    double* dW2 = db1 + kMlpH;
    double* db2 = dW2 + kMlpH * kMlpH;
    double* dW3 = db2 + kMlpH;
    double* db3 = dW3 + 3 * kMlpH;
    float* a1s = sm;
    float* lz2s = sm + kMlpH;
    float* rs = sm + 2 * kMlpH;   // 3 * 64
    float z1 = b1[h];
    z1 = fmaf(__bfloat162float(W1[h * 3]), x[0], z1);
    z1 = fmaf(__bfloat162float(W1[h * 3 + 1]), x[1], z1);
    z1 = fmaf(__bfloat162float(W1[h * 3 + 2]), x[2], z1);
    const float a1 = silu_f(z1);
    a1s[h] = a1;
    sync();
    float z2 = b2[h];
    for (int j = 0; j < kMlpH; ++j) z2 = fmaf(__bfloat162float(W2[h * kMlpH + j]), a1s[j], z2);
    const float a2 = silu_f(z2);
    float la2 = 0.0f;
    for (int m = 0; m < 3; ++m) {
        la2 = fmaf(__bfloat162float(W3[m * kMlpH + h]), (float)lo[m], la2);
        if (dW) dW3[m * kMlpH + h] += lo[m] * (double)a2;
    }
    if (dW && h < 3) db3[h] += lo[h];
    const float sg2 = 1.0f / (1.0f + expf(-z2));
    const float lz2 = la2 * sg2 * (1.0f + z2 * (1.0f - sg2));
    lz2s[h] = lz2;
    sync();
    if (dW) {
        for (int j = 0; j < kMlpH; ++j) dW2[h * kMlpH + j] += (double)lz2 * (double)a1s[j];
        db2[h] += lz2;
    }
    float la1 = 0.0f;
    for (int q = 0; q < kMlpH; ++q) la1 = fmaf(__bfloat162float(W2[q * kMlpH + h]), lz2s[q], la1);
    const float sg1 = 1.0f / (1.0f + expf(-z1));
    const float lz1 = la1 * sg1 * (1.0f + z1 * (1.0f - sg1));
    if (dW) db1[h] += lz1;
    for (int k = 0; k < 3; ++k) {
        if (dW) dW1[h * 3 + k] += (double)lz1 * (double)x[k];
        rs[h * 3 + k] = __bfloat162float(W1[h * 3 + k]) * lz1;
    }
    sync();
    if (h == 0) {
        for (int k = 0; k < 3; ++k) {
            float v = 0.0f;
            for (int q = 0; q < kMlpH; ++q) v += rs[q * 3 + k];
            lx[k] = v;
        }
    }
    sync();
}

// dL/d(C, t, ratio) of the closure inputs from dL/dx (thread 0)
__device__ __forceinline__ void mlp_input_adjoint(const Kin& K, double C, double t, const float lx[3], double* lC, double* lt,
                                  double* lratio)
{
    const double frac = (t < K.t_cool) ? t / K.t_cool : 1.0;
    const double T = K.T0 + (K.T1 - K.T0) * frac;
    const double dTdt = (t < K.t_cool) ? (K.T1 - K.T0) / K.t_cool : 0.0;
    const double cs = K.cs0 + K.cs1 * T + K.cs2 * T * T;
    const double dcs = K.cs1 + 2.0 * K.cs2 * T;
    const double lS = 4.0 * (double)lx[0];
    const double lT = (double)lx[1] / 10.0 - lS * C * dcs / (cs * cs);
    *lC += lS / cs;
    *lt += lT * dTdt;
    *lratio += 1e-6 * (double)lx[2];
}

}  // namespace pbe

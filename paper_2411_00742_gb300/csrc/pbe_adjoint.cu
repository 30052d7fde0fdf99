// Discrete adjoint of the solve (reverse mode through the SSP-RK2 step, the
// gradient the parameter estimation of Sec. 4.1 needs), with checkpointing:
// the forward pass stores the state every K steps; the reverse sweep
// recomputes each K-step segment forward (recording the stage inputs and
// the scalar chain of every step) and then runs the adjoint of the segment
// backwards.
//
// Adjoint of one step (n, C, t) -> (n', C', t'), in reverse order of the
// forward operations:
//   C' = C - kappa (V(n') - V(n))      -> lam_n' += -kappa lam_C' w ...
//   n' = n/2 + n2/2, n2 = n1 + dt L(n1; G_b, B_b)
//   kinetics (G_b, B_b) at (C1, t'),   C1 = C - kappa (V(n1) - V(n))
//   n1 = n + dt L(n; G_a, B_a),        dt from the CFL or the clip branch
//   kinetics (G_a, B_a) at (C, t)
// with L(n) = sum_d G_d D_d(n) + B e_0 / dA, D_d the limited flux
// difference.  (dD/dn)^T lam is a stencil over faces: every face value
// h_f = n_{f-1} + psi(a, b)/2 contributes mu_f = (lam_f - lam_{f-1})/dL
// times its partial derivatives (psi_a = 2 b^2/(a+b)^2, psi_b = 2 a^2/(a+b)^2
// on the branch the forward pass took, 0 otherwise) to the three cells it
// reads.  lam is kept as a stored vector plus pending multiples of the
// moment weight vectors (seeds of output rows, solute-balance terms), which
// the kernels add on the fly.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "pbe_adjoint.cuh"
#include "pbe_internal.h"
#include "pbe_tiles.cuh"

void pbe_set_error_message(int code, const char* msg);  // pbe_api.cu

namespace pbe {

struct AdjS {
    double lC, lt;        // adjoints of C and t at the end of the step being reversed
    double pc[kMaxMom];   // pending: lam_true = lam + sum_k pc[k] W_k
    double pu[kMaxMom];   // pending moment-weight coefficients of u (stage-1 adjoint input)
    double lth[6];        // dL/d(kg1, g1, kg2, g2, kb, b)
    double lCprev, lV0, ldt, ltn;
    unsigned int counter;
};

constexpr int kANT = 256;
constexpr int kAT1 = 512;    // 1-D adjoint tile
constexpr int kATI = 16;     // 2-D adjoint tile
constexpr int kATJ = 32;

// ---------------------------------------------------------------------------
// adjoint stage kernels
//   STAGE 2: lamn' = lam + pending(pc); out = lamn'/2 (lam_prev);
//            u = lam2 + dt (G1b dD1^T + G2b dD2^T) lam2 with lam2 = lamn'/2
//   STAGE 1: lam1 = u + pu W_V; out += lam1 + dt (G1a dD1^T + G2a dD2^T) lam1
// partials: lam_s . D1(nin), lam_s . D2(nin), lam_s at cell 0
// ---------------------------------------------------------------------------
template <int STAGE>
__device__ __forceinline__ double lam_at(const double* lam, const AdjS& A, int vidx, double x1, double x2, double dA,
                                         int ndim)
{
    if (STAGE == 2) {
        double p = ndim == 1 ? poly_weights<1>(A.pc, x1, x2, dA) : poly_weights<2>(A.pc, x1, x2, dA);
        return 0.5 * (*lam + p);
    }
    // STAGE 1: pending terms of u
    (void)vidx;
    return *lam + (ndim == 1 ? poly_weights<1>(A.pu, x1, x2, dA) : poly_weights<2>(A.pu, x1, x2, dA));
}

template <int STAGE>
__global__ void __launch_bounds__(kANT) k_adj1d(const double* __restrict__ nin, const double* __restrict__ lam,
                                                double* out, double* u, AdjS* A, const Scal* __restrict__ recA,
                                                const Scal* __restrict__ recB, Geom g, double* part)
{
    __shared__ double nt[kAT1 + 4];   // cells i0-2 .. i0+T+1
    __shared__ double lt[kAT1 + 3];   // lambda of cells i0-1 .. i0+T+1
    __shared__ double fa[3][kAT1 + 2];  // faces i0 .. i0+T+1
    __shared__ double sh[kANT / 32 * 3];
    __shared__ int flag;
    const int N = g.N1, i0 = blockIdx.x * kAT1;
    const AdjS As = *A;
    const double dt = recA->dt;
    const double G = STAGE == 2 ? recB->G1b : recA->G1a;
    for (int k = threadIdx.x; k < kAT1 + 4; k += kANT) {
        const int i = i0 - 2 + k;
        nt[k] = (i >= 0 && i < N) ? nin[i] : 0.0;
    }
    for (int k = threadIdx.x; k < kAT1 + 3; k += kANT) {
        const int i = i0 - 1 + k;
        double v = 0.0;
        if (i >= 0 && i < N) v = lam_at<STAGE>(lam + i, As, 3, (i + 0.5) * g.d1, 0.0, g.d1, 1);
        lt[k] = v;
    }
    __syncthreads();
    double dot = 0.0;
    for (int k = threadIdx.x; k < kAT1 + 2; k += kANT) {
        const int f = i0 + k;  // face between cells f-1 and f
        if (f > N) { fa[0][k] = fa[1][k] = fa[2][k] = 0.0; continue; }
        // nt index of cell c is c - i0 + 2; lt index of cell c is c - i0 + 1
        const FaceAdj fa_ = face_adj_fast(nt[k], nt[k + 1], nt[k + 2], lt[k], lt[k + 1], g.inv_d1);
        fa[0][k] = fa_.cm2; fa[1][k] = fa_.cm1; fa[2][k] = fa_.c0;
        if (k < kAT1 || (f == N && i0 + kAT1 >= N)) dot += fa_.hmu;   // each face counted by one tile
    }
    __syncthreads();
    double l0 = 0.0;
    for (int c = threadIdx.x; c < kAT1; c += kANT) {
        const int m = i0 + c;
        if (m >= N) break;
        // cell m receives c0 of face m, cm1 of face m+1, cm2 of face m+2 (face index k = f - i0)
        const double jt = fa[2][c] + fa[1][c + 1] + fa[0][c + 2];
        const double ls = lt[c + 1];
        if (m == 0) l0 = ls;
        if (STAGE == 2) {
            out[m] = ls;                       // lam_prev partial = lamn'/2 = lam2
            u[m] = ls + dt * G * jt;
        } else {
            out[m] = out[m] + ls + dt * G * jt;
        }
    }
    double v[3] = {dot, 0.0, l0};
    block_sum<kANT, 3>(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) part[(size_t)blockIdx.x * kMaxMom + k] = v[k];
    if (!last_block(&A->counter, gridDim.x, &flag)) return;
    reduce_partials<kANT, 3>(part, gridDim.x, v, sh);
    if (threadIdx.x == 0) {
        A->counter = 0u;
        part[(size_t)gridDim.x * kMaxMom] = v[0];
        part[(size_t)gridDim.x * kMaxMom + 1] = 0.0;
        part[(size_t)gridDim.x * kMaxMom + 2] = v[2];
    }
}

template <int STAGE>
__global__ void __launch_bounds__(kANT) k_adj2d(const double* __restrict__ nin, const double* __restrict__ lam,
                                                double* out, double* u, AdjS* A, const Scal* __restrict__ recA,
                                                const Scal* __restrict__ recB, Geom g, double* part)
{
    constexpr int TI = kATI, TJ = kATJ;
    constexpr int WN = TJ + 4, WL = TJ + 3;
    __shared__ double nt[(TI + 4) * WN];      // rows i0-2.., cols j0-2..
    __shared__ double lt[(TI + 3) * WL];      // rows i0-1.., cols j0-1..
    __shared__ double f1[3][(TI + 2) * TJ];   // faces along L1 for rows i0..i0+TI+1, columns of the tile
    __shared__ double f2[3][TI * (TJ + 2)];   // faces along L2
    __shared__ double sh[kANT / 32 * 3];
    __shared__ int flag;
    const int N1 = g.N1, N2 = g.N2;
    const int i0 = blockIdx.y * TI, j0 = blockIdx.x * TJ;
    const int nb = gridDim.x * gridDim.y, bid = blockIdx.y * gridDim.x + blockIdx.x;
    const AdjS As = *A;
    const double dt = recA->dt;
    const double G1 = STAGE == 2 ? recB->G1b : recA->G1a;
    const double G2 = STAGE == 2 ? recB->G2b : recA->G2a;
    const double dA = g.d1 * g.d2;
    for (int k = threadIdx.x; k < (TI + 4) * WN; k += kANT) {
        const int r = k / WN, c = k - r * WN;
        const int i = i0 - 2 + r, j = j0 - 2 + c;
        nt[k] = (i >= 0 && i < N1 && j >= 0 && j < N2) ? nin[(size_t)i * N2 + j] : 0.0;
    }
    for (int k = threadIdx.x; k < (TI + 3) * WL; k += kANT) {
        const int r = k / WL, c = k - r * WL;
        const int i = i0 - 1 + r, j = j0 - 1 + c;
        double v = 0.0;
        if (i >= 0 && i < N1 && j >= 0 && j < N2)
            v = lam_at<STAGE>(lam + (size_t)i * N2 + j, As, 8, (i + 0.5) * g.d1, (j + 0.5) * g.d2, dA, 2);
        lt[k] = v;
    }
    __syncthreads();
    double dot1 = 0.0, dot2 = 0.0;
    // faces along L1: face row fr (0..TI+1) is the face between rows i0+fr-1 and i0+fr, column c
    for (int k = threadIdx.x; k < (TI + 2) * TJ; k += kANT) {
        const int fr = k / TJ, c = k - fr * TJ;
        const int f = i0 + fr, j = j0 + c;
        if (f > N1 || j >= N2) { f1[0][k] = f1[1][k] = f1[2][k] = 0.0; continue; }
        // nt row of cell row i is i - i0 + 2; lt row is i - i0 + 1
        const FaceAdj a = face_adj(nt[fr * WN + c + 2], nt[(fr + 1) * WN + c + 2], nt[(fr + 2) * WN + c + 2],
                                   lt[fr * WL + c + 1], lt[(fr + 1) * WL + c + 1], g.inv_d1);
        f1[0][k] = a.cm2; f1[1][k] = a.cm1; f1[2][k] = a.c0;
        if (fr < TI || (f == N1 && i0 + TI >= N1)) dot1 += a.hmu;
    }
    for (int k = threadIdx.x; k < TI * (TJ + 2); k += kANT) {
        const int r = k / (TJ + 2), fc = k - r * (TJ + 2);
        const int i = i0 + r, f = j0 + fc;
        if (i >= N1 || f > N2) { f2[0][k] = f2[1][k] = f2[2][k] = 0.0; continue; }
        const double* nr = nt + (r + 2) * WN;
        const double* lr = lt + (r + 1) * WL;
        const FaceAdj a = face_adj(nr[fc], nr[fc + 1], nr[fc + 2], lr[fc], lr[fc + 1], g.inv_d2);
        f2[0][k] = a.cm2; f2[1][k] = a.cm1; f2[2][k] = a.c0;
        if (fc < TJ || (f == N2 && j0 + TJ >= N2)) dot2 += a.hmu;
    }
    __syncthreads();
    double l0 = 0.0;
    for (int k = threadIdx.x; k < TI * TJ; k += kANT) {
        const int r = k / TJ, c = k - r * TJ;
        const int i = i0 + r, j = j0 + c;
        if (i >= N1 || j >= N2) continue;
        const double j1 = f1[2][r * TJ + c] + f1[1][(r + 1) * TJ + c] + f1[0][(r + 2) * TJ + c];
        const double j2 = f2[2][r * (TJ + 2) + c] + f2[1][r * (TJ + 2) + c + 1] + f2[0][r * (TJ + 2) + c + 2];
        const double ls = lt[(r + 1) * WL + c + 1];
        if (i == 0 && j == 0) l0 = ls;
        const size_t gi = (size_t)i * N2 + j;
        const double jt = dt * (G1 * j1 + G2 * j2);
        if (STAGE == 2) {
            out[gi] = ls;
            u[gi] = ls + jt;
        } else {
            out[gi] = out[gi] + ls + jt;
        }
    }
    double v[3] = {dot1, dot2, l0};
    block_sum<kANT, 3>(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) part[(size_t)bid * kMaxMom + k] = v[k];
    if (!last_block(&A->counter, nb, &flag)) return;
    reduce_partials<kANT, 3>(part, nb, v, sh);
    if (threadIdx.x == 0) {
        A->counter = 0u;
        part[(size_t)nb * kMaxMom] = v[0];
        part[(size_t)nb * kMaxMom + 1] = v[1];
        part[(size_t)nb * kMaxMom + 2] = v[2];
    }
}

// ---------------------------------------------------------------------------
// Scalar steps of the reverse sweep (one thread each).
// ---------------------------------------------------------------------------
// Before the stage-2 adjoint of a step: seeds of the output row the step
// emitted, then the adjoint of C' = C - kappa (V(n') - V(n)).
__global__ void k_adj_begin(AdjS* A, const Scal* recA, const double* seeds, int ncol, int vidx, double kappa)
{
    AdjS a = *A;
    if (recA->clipped) {
        const double* sd = seeds + (size_t)recA->out_idx * ncol;
        for (int k = 0; k < ncol - 2; ++k) a.pc[k] += sd[1 + k];
        a.lC += sd[ncol - 1];
    }
    a.lV0 = kappa * a.lC;
    a.lCprev = a.lC;
    a.pc[vidx] += -kappa * a.lC;
    *A = a;
}

// After the stage-2 adjoint: step length and stage-2 kinetics (at C1, t'),
// then the adjoint of C1 = C - kappa (V(n1) - V(n)).  64 threads.
__global__ void k_adj_mid(AdjS* A, const Scal* recA, const Scal* recB, Kin K, Geom g, const double* tot, int vidx,
                          double* dW)
{
    __shared__ float sm[5 * kMlpH];
    __shared__ float lx[3];
    __shared__ double lo[3];
    __shared__ int run_mlp;
    const double dA = g.ndim == 1 ? g.d1 : g.d1 * g.d2;
    const double P1 = tot[0], P2 = tot[1], P0 = tot[2];
    const double dt = recA->dt;
    if (threadIdx.x == 0) {
        lo[0] = dt * P1 * recB->G1b;
        lo[1] = g.ndim == 2 ? dt * P2 * recB->G2b : 0.0;
        lo[2] = dt * P0 / dA * recB->Bb;
        run_mlp = K.kind == PBE_KINETICS_MLP && !recB->fbb && (recB->G1b > 0.0 || recB->Bb > 0.0);
    }
    __syncthreads();
    if (run_mlp) {
        float x[3];
        mlp_inputs(K, recB->C1, recA->t_new, recB->V1 / recB->M1, x);
        mlp_backward_block64(K, x, lo, dW, sm, lx, BlockSync64());
    }
    if (threadIdx.x != 0) return;
    AdjS a = *A;
    a.ldt = recB->G1b * P1 + recB->G2b * P2 + recB->Bb * P0 / dA;
    double lC1 = 0.0, ltn = a.lt;
    for (int k = 0; k < kMaxMom; ++k) a.pu[k] = 0.0;
    if (K.kind == PBE_KINETICS_MLP && !recB->fbb) {   // else the power law (or the closure's fallback)
        if (run_mlp) {
            double lr = 0.0;
            mlp_input_adjoint(K, recB->C1, recA->t_new, lx, &lC1, &ltn, &lr);
            a.pu[vidx] += lr / recB->M1;
            a.pu[0] += -lr * recB->V1 / (recB->M1 * recB->M1);
        }
    } else {
        kinetics_adjoint(K, recB->C1, recA->t_new, dt * P1, dt * P2, dt * P0 / dA, &lC1, &ltn, a.lth);
    }
    a.ltn = ltn;
    a.lCprev += lC1;
    a.lV0 += K.kappa * lC1;
    a.pu[vidx] += -K.kappa * lC1;
    *A = a;
}

// After the stage-1 adjoint: step length branch, stage-1 kinetics (at C, t),
// and the pending terms of lam for the previous step.  64 threads.
__global__ void k_adj_end(AdjS* A, const Scal* recA, Kin K, Geom g, const double* tot, int vidx, double* dW)
{
    __shared__ float sm[5 * kMlpH];
    __shared__ float lx[3];
    __shared__ double lo[3];
    __shared__ double sl[4];   // ldt, lG1, lG2, lB after the step-length branch
    __shared__ int run_mlp;
    const double dA = g.ndim == 1 ? g.d1 : g.d1 * g.d2;
    const double P1 = tot[0], P2 = tot[1], P0 = tot[2];
    const double dt = recA->dt;
    if (threadIdx.x == 0) {
        const AdjS& a = *A;
        double ldt = a.ldt + recA->G1a * P1 + recA->G2a * P2 + recA->Ba * P0 / dA;
        double lG1 = dt * P1, lG2 = dt * P2;
        if (!recA->clipped) {
            ldt += a.ltn;
            double R = recA->G1a / g.d1;
            if (g.ndim == 2) R = R + recA->G2a / g.d2;
            const double dR = -K.cfl / (R * R) * ldt;
            lG1 += dR / g.d1;
            if (g.ndim == 2) lG2 += dR / g.d2;
        }
        sl[0] = ldt; sl[1] = lG1; sl[2] = lG2; sl[3] = dt * P0 / dA;
        lo[0] = lG1 * recA->G1a;
        lo[1] = g.ndim == 2 ? lG2 * recA->G2a : 0.0;
        lo[2] = sl[3] * recA->Ba;
        run_mlp = K.kind == PBE_KINETICS_MLP && !recA->fba && (recA->G1a > 0.0 || recA->Ba > 0.0);
    }
    __syncthreads();
    if (run_mlp) {
        float x[3];
        mlp_inputs(K, recA->C, recA->t, recA->V0 / recA->M0, x);
        mlp_backward_block64(K, x, lo, dW, sm, lx, BlockSync64());
    }
    if (threadIdx.x != 0) return;
    AdjS a = *A;
    double ltp = recA->clipped ? -sl[0] : a.ltn;
    double lC = a.lCprev;
    for (int k = 0; k < kMaxMom; ++k) a.pc[k] = 0.0;
    if (K.kind == PBE_KINETICS_MLP && !recA->fba) {   // else the power law (or the closure's fallback)
        if (run_mlp) {
            double lr = 0.0;
            mlp_input_adjoint(K, recA->C, recA->t, lx, &lC, &ltp, &lr);
            a.pc[vidx] += lr / recA->M0;
            a.pc[0] += -lr * recA->V0 / (recA->M0 * recA->M0);
        }
    } else {
        kinetics_adjoint(K, recA->C, recA->t, sl[1], sl[2], sl[3], &lC, &ltp, a.lth);
    }
    a.lC = lC;
    a.lt = ltp;
    a.pc[vidx] += a.lV0;
    *A = a;
}

// Seeds of a row emitted at the start time (before any step).
__global__ void k_adj_row0(AdjS* A, const double* seeds, int ncol)
{
    for (int k = 0; k < ncol - 2; ++k) A->pc[k] += seeds[1 + k];
    A->lC += seeds[ncol - 1];
}

// lam0 = lam + pending moment-weight terms.
template <int NDIM>
__global__ void k_adj_final(double* lam, const AdjS* A, Geom g)
{
    __shared__ double pc[kMaxMom];
    if (threadIdx.x < kMaxMom) pc[threadIdx.x] = A->pc[threadIdx.x];
    __syncthreads();
    const long long ncell = (long long)g.N1 * g.N2;
    const double dA = g.ndim == 1 ? g.d1 : g.d1 * g.d2;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c / g.N2), j = (int)(c % g.N2);
        lam[c] += poly_weights<NDIM>(pc, (i + 0.5) * g.d1, (j + 0.5) * g.d2, dA);
    }
}

static int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

int adj_blocks(const Geom& g) { return g.ndim == 1 ? cdiv(g.N1, kAT1) : cdiv(g.N1, kATI) * cdiv(g.N2, kATJ); }

cudaError_t launch_adj_stage(int stage, const Geom& g, const double* nin, const double* lam, double* out, double* u,
                             AdjS* A, const Scal* recA, const Scal* recB, double* part, cudaStream_t st)
{
    if (g.ndim == 1) {
        const int nb = cdiv(g.N1, kAT1);
        if (stage == 2) k_adj1d<2><<<nb, kANT, 0, st>>>(nin, lam, out, u, A, recA, recB, g, part);
        else k_adj1d<1><<<nb, kANT, 0, st>>>(nin, lam, out, u, A, recA, recB, g, part);
    } else {
        dim3 grid(cdiv(g.N2, kATJ), cdiv(g.N1, kATI));
        if (stage == 2) k_adj2d<2><<<grid, kANT, 0, st>>>(nin, lam, out, u, A, recA, recB, g, part);
        else k_adj2d<1><<<grid, kANT, 0, st>>>(nin, lam, out, u, A, recA, recB, g, part);
    }
    return cudaGetLastError();
}

}  // namespace pbe

using namespace pbe;

namespace {

pbe_status afail(pbe_status code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    pbe_set_error_message(code, buf);
    return code;
}

#define ATRY(call)                                                                                     \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) { rc = afail(PBE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); goto done; } \
    } while (0)

}  // namespace

extern "C" pbe_status pbe_vjp(pbe_grid* g, const double* t_out, int n_out, const double* seeds_in, int seeds_mem,
                              int checkpoint_every, double* dL_dtheta, double* dL_dn0, double* dL_dC0, double* rows,
                              int mem, double* dL_dweights)
{
    if (!g || !t_out || !seeds_in || !dL_dtheta) return afail(PBE_EINVAL, "null argument");
    if (n_out < 1) return afail(PBE_EINVAL, "n_out must be >= 1");
    if (checkpoint_every < 1) return afail(PBE_EINVAL, "checkpoint_every must be >= 1");
    if (!g->has_kin || !g->has_state) return afail(PBE_ESTATE, "set kinetics and state before pbe_vjp");
    if (g->kin.scheme != PBE_SCHEME_SSPRK2 || g->kin.growth_form == 1 || g->kin.solubility_form != 0)
        return afail(PBE_EINVAL, "the adjoint differentiates the SSP-RK2 scheme with power-law kinetics, the "
                                 "polynomial growth law or the closure");
    const bool persistent = g->path == PBE_PATH_FUSED && fused_supported(g);
    if (g->kin.growth_form == 2 && !persistent)
        return afail(PBE_EINVAL, "the polynomial growth law is differentiated on the fused path (pbe_set_path)");
    if (!(t_out[0] >= g->t_host)) return afail(PBE_EINVAL, "t_out[0] precedes the current time");
    for (int j = 1; j < n_out; ++j)
        if (!(t_out[j] > t_out[j - 1]) || !std::isfinite(t_out[j])) return afail(PBE_EINVAL, "t_out must increase");
    if (persistent)
        return vjp_persistent(g, t_out, n_out, seeds_in, seeds_mem, checkpoint_every, dL_dtheta, dL_dn0, dL_dC0,
                              rows, mem, dL_dweights);
    const int ncol = g->geo.ndim == 1 ? 6 : 12, vidx = g->geo.ndim == 1 ? 3 : 8;
    const size_t nc = g->ncell, sz = nc * sizeof(double);
    const int K = checkpoint_every;
    const double t0 = g->t_host;
    cudaStream_t st = g->stream;
    pbe_status rc = PBE_OK;
    std::vector<double*> ckpt_n;
    std::vector<Scal*> ckpt_S;
    double *seg_n = nullptr, *seg_n1 = nullptr, *lam = nullptr, *lam2 = nullptr, *u = nullptr, *seeds = nullptr;
    double *fin_n = nullptr, *apart = nullptr, *dW = nullptr;
    Scal *recA = nullptr, *recB = nullptr, *fin_S = nullptr;
    AdjS* A = nullptr;
    long long total = 0;
    int nck = 0;
    const int nb = adj_blocks(g->geo);
    AdjS ha;
    double* tot;
    {
        int prev_dev = -1;
        cudaGetDevice(&prev_dev);
        if (prev_dev != g->device) cudaSetDevice(g->device);
    }
    ATRY(cudaMalloc(&seg_n, sz * K));
    ATRY(cudaMalloc(&seg_n1, sz * K));
    ATRY(cudaMalloc(&recA, sizeof(Scal) * K));
    ATRY(cudaMalloc(&recB, sizeof(Scal) * K));
    ATRY(cudaMalloc(&lam, sz));
    ATRY(cudaMalloc(&lam2, sz));
    ATRY(cudaMalloc(&u, sz));
    ATRY(cudaMalloc(&fin_n, sz));
    ATRY(cudaMalloc(&fin_S, sizeof(Scal)));
    ATRY(cudaMalloc(&seeds, sizeof(double) * ncol * n_out));
    ATRY(cudaMalloc(&A, sizeof(AdjS)));
    ATRY(cudaMalloc(&apart, sizeof(double) * kMaxMom * (nb + 1)));
    ATRY(cudaMalloc(&dW, sizeof(double) * kMlpNW));
    ATRY(cudaMemsetAsync(dW, 0, sizeof(double) * kMlpNW, st));
    tot = apart + (size_t)nb * kMaxMom;
    ATRY(cudaMemcpyAsync(seeds, seeds_in, sizeof(double) * ncol * n_out,
                         seeds_mem == PBE_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    // ---- forward with checkpoints every K steps ----
    {
        const pbe_status ps = prepare_tout(g, t_out, n_out);
        if (ps != PBE_OK) { rc = ps; goto done; }
    }
    ATRY(launch_prologue(g, n_out, g->max_steps, nullptr));
    for (;;) {
        double* cn;
        Scal* cs;
        ATRY(cudaMalloc(&cn, sz));
        ATRY(cudaMalloc(&cs, sizeof(Scal)));
        ckpt_n.push_back(cn);
        ckpt_S.push_back(cs);
        ATRY(cudaMemcpyAsync(cn, g->d_n, sz, cudaMemcpyDeviceToDevice, st));
        ATRY(cudaMemcpyAsync(cs, g->d_S, sizeof(Scal), cudaMemcpyDeviceToDevice, st));
        for (int k = 0; k < K; ++k) ATRY(launch_plain_step(g, false, 0));
        ATRY(cudaMemcpyAsync(g->h_S, g->d_S, sizeof(Scal), cudaMemcpyDeviceToHost, st));
        ATRY(cudaStreamSynchronize(st));
        if (g->h_S->done) break;
        if ((long long)ckpt_n.size() * K > g->max_steps + K) { rc = afail(PBE_ETIMEOUT, "step budget exhausted"); goto done; }
    }
    if (g->h_S->status != PBE_OK) { rc = afail(g->h_S->status, "forward solve failed with status %d", g->h_S->status); goto done; }
    total = g->h_S->steps;
    nck = (int)((total + K - 1) / K);
    if (rows) ATRY(cudaMemcpyAsync(rows, g->d_rows, sizeof(double) * ncol * n_out,
                                   mem == PBE_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    ATRY(cudaMemcpyAsync(fin_n, g->d_n, sz, cudaMemcpyDeviceToDevice, st));
    ATRY(cudaMemcpyAsync(fin_S, g->d_S, sizeof(Scal), cudaMemcpyDeviceToDevice, st));
    // ---- reverse sweep ----
    ATRY(cudaMemsetAsync(A, 0, sizeof(AdjS), st));
    ATRY(cudaMemsetAsync(lam, 0, sz, st));
    for (int c = nck - 1; c >= 0; --c) {
        const long long s0 = (long long)c * K, s1 = std::min(s0 + K, total);
        ATRY(cudaMemcpyAsync(g->d_n, ckpt_n[c], sz, cudaMemcpyDeviceToDevice, st));
        ATRY(cudaMemcpyAsync(g->d_S, ckpt_S[c], sizeof(Scal), cudaMemcpyDeviceToDevice, st));
        for (long long s = s0; s < s1; ++s) {
            const long long q = s - s0;
            ATRY(cudaMemcpyAsync(recA + q, g->d_S, sizeof(Scal), cudaMemcpyDeviceToDevice, st));
            ATRY(cudaMemcpyAsync(seg_n + q * nc, g->d_n, sz, cudaMemcpyDeviceToDevice, st));
            // one forward step, with the stage-1 output and scalars recorded
            {
                const Geom& geo = g->geo;
                (void)geo;
            }
            ATRY(launch_plain_stage(g, 1));
            ATRY(cudaMemcpyAsync(seg_n1 + q * nc, g->d_n1, sz, cudaMemcpyDeviceToDevice, st));
            ATRY(cudaMemcpyAsync(recB + q, g->d_S, sizeof(Scal), cudaMemcpyDeviceToDevice, st));
            ATRY(launch_plain_stage(g, 2));
        }
        for (long long s = s1 - 1; s >= s0; --s) {
            const long long q = s - s0;
            k_adj_begin<<<1, 1, 0, st>>>(A, recA + q, seeds, ncol, vidx, g->kin.kappa);
            ATRY(cudaGetLastError());
            ATRY(launch_adj_stage(2, g->geo, seg_n1 + q * nc, lam, lam2, u, A, recA + q, recB + q, apart, st));
            k_adj_mid<<<1, kMlpH, 0, st>>>(A, recA + q, recB + q, g->kin, g->geo, tot, vidx, dW);
            ATRY(cudaGetLastError());
            ATRY(launch_adj_stage(1, g->geo, seg_n + q * nc, u, lam2, nullptr, A, recA + q, recB + q, apart, st));
            k_adj_end<<<1, kMlpH, 0, st>>>(A, recA + q, g->kin, g->geo, tot, vidx, dW);
            ATRY(cudaGetLastError());
            std::swap(lam, lam2);
        }
    }
    if (t_out[0] == t0) {
        k_adj_row0<<<1, 1, 0, st>>>(A, seeds, ncol);
        ATRY(cudaGetLastError());
    }
    if (g->geo.ndim == 1)
        k_adj_final<1><<<std::max(1, std::min(1024, cdiv(nc, 256))), 256, 0, st>>>(lam, A, g->geo);
    else
        k_adj_final<2><<<std::max(1, std::min(1024, cdiv(nc, 256))), 256, 0, st>>>(lam, A, g->geo);
    ATRY(cudaGetLastError());
    if (dL_dn0) ATRY(cudaMemcpyAsync(dL_dn0, lam, sz, mem == PBE_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    ATRY(cudaMemcpyAsync(&ha, A, sizeof(AdjS), cudaMemcpyDeviceToHost, st));
    // leave the grid at the end of the solve
    ATRY(cudaMemcpyAsync(g->d_n, fin_n, sz, cudaMemcpyDeviceToDevice, st));
    ATRY(cudaMemcpyAsync(g->d_S, fin_S, sizeof(Scal), cudaMemcpyDeviceToDevice, st));
    ATRY(cudaMemcpyAsync(g->h_S, fin_S, sizeof(Scal), cudaMemcpyDeviceToHost, st));
    ATRY(cudaStreamSynchronize(st));
    g->C_host = g->h_S->C;
    g->t_host = g->h_S->t;
    if (dL_dweights) ATRY(cudaMemcpy(dL_dweights, dW, sizeof(double) * kMlpNW, cudaMemcpyDeviceToHost));
    for (int k = 0; k < 6; ++k) dL_dtheta[k] = ha.lth[k];
    if (dL_dC0) *dL_dC0 = ha.lC;
    if (!std::isfinite(ha.lth[0]) || !std::isfinite(ha.lth[1]) || !std::isfinite(ha.lth[4]) || !std::isfinite(ha.lth[5]))
        rc = afail(PBE_ENONFINITE, "non-finite gradient");
done:
    cudaStreamSynchronize(st);
    for (double* p : ckpt_n) cudaFree(p);
    for (Scal* p : ckpt_S) cudaFree(p);
    cudaFree(seg_n); cudaFree(seg_n1); cudaFree(recA); cudaFree(recB); cudaFree(lam); cudaFree(lam2); cudaFree(u);
    cudaFree(fin_n); cudaFree(fin_S); cudaFree(seeds); cudaFree(A); cudaFree(apart); cudaFree(dW);
    return rc;
}

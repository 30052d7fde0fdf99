// Persistent discrete adjoint of one grid (the gradient of Sec. 4.1 by
// reverse mode with checkpointing), one cooperative launch per gradient:
//
//  1. forward pass: the SSP-RK2 solve, storing the state every K steps
//     (checkpoints) and recording, for the steps of the current K-step
//     segment, the stage-1 input n^k, the stage-1 output n1 and the scalar
//     chain (kinetics, step length, solute balance, ln s of both kinetics);
//  2. reverse sweep, segment by segment from the last: every segment but the
//     last is recomputed from its checkpoint (the last one is still recorded
//     from the forward pass), then its steps are reversed - the stage-2
//     adjoint, the step-length and stage-2 kinetics backward, the stage-1
//     adjoint, the stage-1 kinetics backward;
//  3. lam0 = dL/dn0 with the pending moment-weight terms added, dL/dtheta
//     and dL/dC0.
//
// Every block owns fixed tiles of the grid (2-D: ti x 32 cells, 1-D: 512
// cells) for the whole launch and runs a private copy of the scalar chains
// (forward and adjoint), so the only device-wide exchanges are the two
// barriers of every forward or reverse step.  Forward barriers carry the
// volume moment as an exact fixed-point sum (barrier_sum); reverse barriers
// are arrival counts after which every block sums the blocks' partial dot
// products in a fixed order (deterministic).  A grid that fits one tile runs
// in one block, where the barriers are __syncthreads.  Every wait is bounded
// (PBE_ETIMEOUT, never a hang).
//
// The reverse arithmetic is that of the per-stage adjoint kernels
// (pbe_adjoint.cu) for the fast forward path (Newton-refined face
// quotients): (dD/dn)^T lam is a stencil over faces, face f contributing
// mu_f = (lam_f - lam_{f-1})/dL times dh/dn to the cells f-2, f-1, f, with
// dh/dn = (-q^2, 2q, (1-q)^2), q = b/(a+b) on the limited branch the forward
// took, (0, 1, 0) otherwise; lam is kept as a vector plus pending multiples
// of moment-weight vectors (output seeds and solute-balance terms).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#include "pbe_adjoint.cuh"
#include "pbe_chain.cuh"
#include "pbe_internal.h"
#include "pbe_sync.cuh"
#include "pbe_tiles.cuh"

namespace pbe {

constexpr int kPNT = 256;   // threads per block
constexpr int kPT1 = 512;   // largest 1-D tile (cells)
constexpr int kPT1Min = 64; // smallest 1-D tile: small grids spread over several blocks
constexpr int kPTI = 16;    // largest 2-D tile height
constexpr int kPTJ = 32;    // 2-D tile width
constexpr int kStatusGrow = -2;   // the checkpoint store is full: the host grows it and runs again

// adjoint scalars of the reverse sweep (every block keeps an identical copy)
struct RevS {
    double lC, lt;            // adjoints of C and t at the end of the step being reversed
    double pc[kMaxMom];       // pending terms of lam: lam_true = lam + sum_k pc[k] W_k
    double pv, p0;            // pending terms of u (stage-1 input): pv W_V + p0 W_0
    double lth[6];            // dL/d(kg1, g1, kg2, g2, kb, b)
    double lCprev, lV0, ldt, ltn;
    double sum[3];            // the last reverse barrier's sums: lam . D1(n), lam . D2(n), lam at cell 0
    double plG1, plG2, ps, pL;  // polynomial growth law: dL/dG_m, s and ln s of the stage just reversed
};

struct AdjOut {
    double lth[6];
    double lC;
    long long steps;
    long long nrows;    // closure evaluations recorded in mrows
    int status;
    int row_first, row_end;
};

struct AdjP {
    double* n;          // initial state (stage-1 input of step 0); receives the final state
    double* fin;        // the final state while the reverse sweep runs
    Scal* S;            // scalars prepared by the prologue; receives the final ones
    Kin K;
    Geom g;
    const double* t_out;
    double* rows;
    double* rowpart;    // [row][block][NM]
    double* seg_n;      // K-1 slots: state at the start of step q = 1..K-1 of the current segment
    double* seg_n1;     // K slots: stage-1 output of step q
    double* ck;         // ck_cap slots: the state after segment c (checkpoint c + 1)
    Scal* recA;         // K: scalars at the start of step q (kinetics a, dt)
    Scal* recB;         // K: scalars after the stage-1 close (C1, kinetics b)
    Scal* ckS;          // ck_cap + 1: scalars at the start of segment c
    double* lamA;
    double* lamB;
    double* u;
    double* part;       // [2][G][4] block partials of the reverse barriers and the mu0 sums
    const double* seeds;
    double* dW;         // learned closure: dL/dweights (fp64), accumulated by block 0
    double* dpoly;      // polynomial growth law: dL/da (ndim x npoly), accumulated by block 0
    float* mrows;       // learned closure: block 0 records one row (x0, x1, x2, lo0, lo1, lo2) per
    long long mrows_cap;    // differentiated evaluation, for the weight-gradient kernel (null: none)
    AdjOut* out;
    unsigned long long* acc;
    size_t nc;
    int Kc, ck_cap, n_out, ncol;
    int ntiles, tiles_x, ti;
    int t1;             // 1-D tile cells (kPT1Min .. kPT1)
    int fwd_only;       // 1: the solve only (state in n and fin, stage-1 output in u, no records)
    long long wait_limit;
    double t0;
};

// ---- shared memory of one block --------------------------------------------
struct FwdSm1 {
    double tile[kPT1 + 3];
    double h[kPT1 + 1];
};
struct FwdSm2 {
    double tile[(kPTI + 3) * (kPTJ + 3)];
    double h1[(kPTI + 1) * kPTJ];
    double h2[kPTI * (kPTJ + 1)];
};
struct RevSm1 {
    double nt[kPT1 + 4];        // cells i0-2 .. i0+T+1
    double lt[kPT1 + 3];        // lambda of cells i0-1 .. i0+T+1
    double fa[3][kPT1 + 2];     // faces i0 .. i0+T+1
};
struct RevSm2 {
    double nt[(kPTI + 4) * (kPTJ + 4)];
    double lt[(kPTI + 3) * (kPTJ + 3)];
    double f1[3][(kPTI + 2) * kPTJ];
    double f2[3][kPTI * (kPTJ + 2)];
};
union TileSm {
    FwdSm1 f1;
    FwdSm2 f2;
    RevSm1 r1;
    RevSm2 r2;
};

// state at the start of step q of segment c
__device__ __forceinline__ double* st_ptr(const AdjP& P, int c, int q)
{
    if (q == 0) return c == 0 ? P.n : P.ck + (size_t)(c - 1) * P.nc;
    return P.seg_n + (size_t)(q - 1) * P.nc;
}

template <int NDIM>
__device__ __forceinline__ void tile_org(const AdjP& P, int t, int& i0, int& j0)
{
    if (NDIM == 1) { i0 = t * P.t1; j0 = 0; }
    else { i0 = (t / P.tiles_x) * P.ti; j0 = (t % P.tiles_x) * kPTJ; }
}

// ---- forward stage of one tile ---------------------------------------------
// STAGE 1: out = in + dt L(in); STAGE 2: out = old/2 + (in + dt L(in))/2.
// Face values by the Newton-refined quotient (face_value<true>).  Moments of
// `out`: the volume moment always, mu0 when m0, all when moms.
template <int STAGE>
__device__ __forceinline__ void fwd_tile1d(const double* in, const double* old, double* out, int i0, int T,
                                           const Geom& g, const StageCoef& sc, bool moms, bool m0,
                                           double (&m)[kMaxMom], FwdSm1& s)
{
    const int N = g.N1;
    for (int k = threadIdx.x; k < T + 3; k += kPNT) {
        const int gi = i0 - 2 + k;
        s.tile[k] = (gi >= 0 && gi < N) ? __ldcg(in + gi) : 0.0;
    }
    __syncthreads();
    for (int f = threadIdx.x; f <= T; f += kPNT) s.h[f] = face_value<true>(s.tile[f], s.tile[f + 1], s.tile[f + 2]);
    __syncthreads();
    for (int c = threadIdx.x; c < T; c += kPNT) {
        const int i = i0 + c;
        if (i >= N) break;
        double v = s.tile[c + 2] + sc.c1 * (s.h[c] - s.h[c + 1]);
        if (i == 0) v += sc.src;
        if (STAGE == 2) v = 0.5 * __ldcg(old + i) + 0.5 * v;
        out[i] = v;
        const double x = (i + 0.5) * g.d1, w = v * g.d1;
        if (moms) { m[0] += w; m[1] += x * w; m[2] += x * x * w; }
        else if (m0) m[0] += w;
        m[3] += x * x * x * w;
    }
    __syncthreads();
}

template <int STAGE>
__device__ __forceinline__ void fwd_tile2d(const double* in, const double* old, double* out, int i0, int j0, int ti,
                                           const Geom& g, const StageCoef& sc, bool moms, bool m0,
                                           double (&m)[kMaxMom], FwdSm2& s)
{
    constexpr int W = kPTJ + 3;
    const int N1 = g.N1, N2 = g.N2;
    for (int k = threadIdx.x; k < (ti + 3) * W; k += kPNT) {
        const int r = k / W, c = k - r * W;
        const int gi = i0 - 2 + r, gj = j0 - 2 + c;
        s.tile[k] = (gi >= 0 && gi < N1 && gj >= 0 && gj < N2) ? __ldcg(in + (size_t)gi * N2 + gj) : 0.0;
    }
    __syncthreads();
    const int n1f = (ti + 1) * kPTJ;
    for (int k = threadIdx.x; k < n1f + ti * (kPTJ + 1); k += kPNT) {
        if (k < n1f) {
            const int f = k / kPTJ, c = k - f * kPTJ;
            s.h1[k] = face_value<true>(s.tile[f * W + c + 2], s.tile[(f + 1) * W + c + 2], s.tile[(f + 2) * W + c + 2]);
        } else {
            const int kk = k - n1f, r = kk / (kPTJ + 1), f = kk - r * (kPTJ + 1);
            const double* row = s.tile + (r + 2) * W;
            s.h2[kk] = face_value<true>(row[f], row[f + 1], row[f + 2]);
        }
    }
    __syncthreads();
    const double area = g.d1 * g.d2;
    for (int k = threadIdx.x; k < ti * kPTJ; k += kPNT) {
        const int r = k / kPTJ, c = k - r * kPTJ;
        const int i = i0 + r, j = j0 + c;
        if (i >= N1 || j >= N2) continue;
        double v = s.tile[(r + 2) * W + c + 2] + sc.c1 * (s.h1[r * kPTJ + c] - s.h1[(r + 1) * kPTJ + c]) +
                   sc.c2 * (s.h2[r * (kPTJ + 1) + c] - s.h2[r * (kPTJ + 1) + c + 1]);
        if (i == 0 && j == 0) v += sc.src;
        const size_t gidx = (size_t)i * N2 + j;
        if (STAGE == 2) v = 0.5 * __ldcg(old + gidx) + 0.5 * v;
        out[gidx] = v;
        const double x1 = (i + 0.5) * g.d1, x2 = (j + 0.5) * g.d2;
        const double w = v * area, x1w = x1 * w, x2w = x2 * w;
        m[8] += x1 * x2 * x2w;
        if (moms) {
            m[0] += w; m[1] += x1w; m[2] += x2w;
            m[3] += x1 * x1w; m[4] += x1 * x2w; m[5] += x2 * x2w;
            m[6] += x1 * x1 * x1w; m[7] += x1 * x1 * x2w; m[9] += x2 * x2 * x2w;
        } else if (m0) {
            m[0] += w;
        }
    }
    __syncthreads();
}

// ---- reverse stage of one tile ---------------------------------------------

// STAGE 2: lam2 = (lam + sum_k pc[k] W_k)/2; out = lam2 (the Runge-Kutta
//          average's share of lam_n); u = lam2 + dt (G1 dD1^T + G2 dD2^T) lam2
//          over the stage-1 output nin.
// STAGE 1: lam1 = u + pv W_V + p0 W_0; out += lam1 + dt (G1 dD1^T + G2 dD2^T)
//          lam1 over the stage-1 input nin.
// acc += (lam_s . D1(nin), lam_s . D2(nin), lam_s at cell 0) of the tile.
// own (one-tile blocks, else null): stage 2 keeps lam2 of the tile's cells
// there, stage 1 reads it instead of `out`.
template <int STAGE>
__device__ __forceinline__ void rev_tile1d(const double* nin, const double* lam, double* out, double* u, int i0,
                                           int T, const Geom& g, double dt, double G, const RevS& R, double (&acc)[3],
                                           double* own, RevSm1& s)
{
    const int N = g.N1;
    for (int k = threadIdx.x; k < T + 4; k += kPNT) {
        const int i = i0 - 2 + k;
        s.nt[k] = (i >= 0 && i < N) ? __ldcg(nin + i) : 0.0;
    }
    for (int k = threadIdx.x; k < T + 3; k += kPNT) {
        const int i = i0 - 1 + k;
        double v = 0.0;
        if (i >= 0 && i < N) {
            const double x = (i + 0.5) * g.d1;
            v = __ldcg(lam + i);
            if (STAGE == 2) v = 0.5 * (v + poly_weights<1>(R.pc, x, 0.0, g.d1));
            else v += (R.p0 + R.pv * (x * x * x)) * g.d1;
        }
        s.lt[k] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < T + 2; k += kPNT) {
        const int f = i0 + k;   // face between cells f-1 and f
        if (f > N) { s.fa[0][k] = s.fa[1][k] = s.fa[2][k] = 0.0; continue; }
        const FaceAdj fa = face_adj_fast(s.nt[k], s.nt[k + 1], s.nt[k + 2], s.lt[k], s.lt[k + 1], g.inv_d1);
        s.fa[0][k] = fa.cm2; s.fa[1][k] = fa.cm1; s.fa[2][k] = fa.c0;
        if (k < T || (f == N && i0 + T >= N)) acc[0] += fa.hmu;   // each face counted by one tile
    }
    __syncthreads();
    for (int c = threadIdx.x; c < T; c += kPNT) {
        const int m = i0 + c;
        if (m >= N) break;
        // cell m receives c0 of face m, cm1 of face m+1 and cm2 of face m+2
        const double jt = s.fa[2][c] + s.fa[1][c + 1] + s.fa[0][c + 2];
        const double ls = s.lt[c + 1];
        if (m == 0) acc[2] += ls;
        if (STAGE == 2) {
            out[m] = ls;
            if (own) own[c] = ls;
            u[m] = fma(dt * G, jt, ls);
        } else {
            out[m] = (own ? own[c] : __ldcg(out + m)) + ls + (dt * G) * jt;
        }
    }
    __syncthreads();
}

template <int STAGE>
__device__ __forceinline__ void rev_tile2d(const double* nin, const double* lam, double* out, double* u, int i0,
                                           int j0, int ti, const Geom& g, double dt, double G1, double G2,
                                           const RevS& R, double (&acc)[3], double* own, RevSm2& s)
{
    constexpr int TJ = kPTJ, WN = TJ + 4, WL = TJ + 3;
    const int N1 = g.N1, N2 = g.N2;
    const double dA = g.d1 * g.d2;
    for (int k = threadIdx.x; k < (ti + 4) * WN; k += kPNT) {
        const int r = k / WN, c = k - r * WN;
        const int i = i0 - 2 + r, j = j0 - 2 + c;
        s.nt[k] = (i >= 0 && i < N1 && j >= 0 && j < N2) ? __ldcg(nin + (size_t)i * N2 + j) : 0.0;
    }
    for (int k = threadIdx.x; k < (ti + 3) * WL; k += kPNT) {
        const int r = k / WL, c = k - r * WL;
        const int i = i0 - 1 + r, j = j0 - 1 + c;
        double v = 0.0;
        if (i >= 0 && i < N1 && j >= 0 && j < N2) {
            const double x1 = (i + 0.5) * g.d1, x2 = (j + 0.5) * g.d2;
            v = __ldcg(lam + (size_t)i * N2 + j);
            if (STAGE == 2) v = 0.5 * (v + poly_weights<2>(R.pc, x1, x2, dA));
            else v += (R.p0 + R.pv * (x1 * x2 * x2)) * dA;
        }
        s.lt[k] = v;
    }
    __syncthreads();
    // faces along L1: face row fr (0..ti+1) between cell rows i0+fr-1 and i0+fr;
    // then faces along L2: row r, face column fc (0..TJ+1) between columns j0+fc-1 and j0+fc
    const int n1f = (ti + 2) * TJ;
    for (int k = threadIdx.x; k < n1f + ti * (TJ + 2); k += kPNT) {
        if (k < n1f) {
            const int fr = k / TJ, c = k - fr * TJ;
            const int f = i0 + fr, j = j0 + c;
            if (f > N1 || j >= N2) { s.f1[0][k] = s.f1[1][k] = s.f1[2][k] = 0.0; continue; }
            const FaceAdj a = face_adj_fast(s.nt[fr * WN + c + 2], s.nt[(fr + 1) * WN + c + 2],
                                            s.nt[(fr + 2) * WN + c + 2], s.lt[fr * WL + c + 1],
                                            s.lt[(fr + 1) * WL + c + 1], g.inv_d1);
            s.f1[0][k] = a.cm2; s.f1[1][k] = a.cm1; s.f1[2][k] = a.c0;
            if (fr < ti || (f == N1 && i0 + ti >= N1)) acc[0] += a.hmu;
        } else {
            const int kk = k - n1f, r = kk / (TJ + 2), fc = kk - r * (TJ + 2);
            const int i = i0 + r, f = j0 + fc;
            if (i >= N1 || f > N2) { s.f2[0][kk] = s.f2[1][kk] = s.f2[2][kk] = 0.0; continue; }
            const double* nr = s.nt + (r + 2) * WN;
            const double* lr = s.lt + (r + 1) * WL;
            const FaceAdj a = face_adj_fast(nr[fc], nr[fc + 1], nr[fc + 2], lr[fc], lr[fc + 1], g.inv_d2);
            s.f2[0][kk] = a.cm2; s.f2[1][kk] = a.cm1; s.f2[2][kk] = a.c0;
            if (fc < TJ || (f == N2 && j0 + TJ >= N2)) acc[1] += a.hmu;
        }
    }
    __syncthreads();
    const double c1 = dt * G1, c2 = dt * G2;
    for (int k = threadIdx.x; k < ti * TJ; k += kPNT) {
        const int r = k / TJ, c = k - r * TJ;
        const int i = i0 + r, j = j0 + c;
        if (i >= N1 || j >= N2) continue;
        const double j1 = s.f1[2][r * TJ + c] + s.f1[1][(r + 1) * TJ + c] + s.f1[0][(r + 2) * TJ + c];
        const double j2 = s.f2[2][r * (TJ + 2) + c] + s.f2[1][r * (TJ + 2) + c + 1] + s.f2[0][r * (TJ + 2) + c + 2];
        const double ls = s.lt[(r + 1) * WL + c + 1];
        if (i == 0 && j == 0) acc[2] += ls;
        const size_t gi = (size_t)i * N2 + j;
        const double jt = fma(c1, j1, c2 * j2);
        if (STAGE == 2) {
            out[gi] = ls;
            if (own) own[k] = ls;
            u[gi] = ls + jt;
        } else {
            out[gi] = (own ? own[k] : __ldcg(out + gi)) + ls + jt;
        }
    }
    __syncthreads();
}

// ---- block state --------------------------------------------------------------
struct BlockSm {
    TileSm t;        // also the staging area of block_sum_staged
    Scal s;          // forward scalar chain (identical in every block)
    Scal sfin;       // the scalars at the end of the forward pass
    Scal sA, sB;     // records of the step being reversed
    Scal nA, nB;     // the next reversed step's records, prefetched during the stage-2 cells
    double own[kPT1];   // one-tile blocks: lam2 of the own cells from stage 2 to stage 1
    RevS R;
    StageCoef sc;    // coefficients of the coming forward stage
    double red[kMaxMom];   // block sums of block_sum_staged
    long long wsum[kPNT / 32];
    double psum[4];  // this block's partials (read directly in one-block launches)
    double ik[3];    // 1/kg1, 1/kg2, 1/kb (0 where the prefactor is 0)
    double inv_dA, inv_cfl;
    float mlp_sm[5 * kMlpH];
    float mlp_lx[3];
    double mlp_lo[3];
    double vtot;
    int par;         // parity of the last forward barrier (its block partials)
    int run_mlp, fail;
    long long nrow;  // closure rows recorded (block 0)
};

struct Bar64 {   // named barrier over threads 0..63 (the closure backward)
    __device__ __forceinline__ void operator()() const { asm volatile("bar.sync 5, 64;" ::: "memory"); }
};

// Block sum of NV values (deterministic): every thread's values go to shared
// memory, then warp k sums value k (eight values a lane in block order, then
// a butterfly) - NV warps x 13 FP64 additions instead of the 8 x 5 NV of a
// shuffle tree in every warp, which on GB300 would hold the SM's FP64 pipe
// for ~16 cycles each.  `sh` holds kPNT * NV doubles; the sums land in
// out[0..NV) (shared), valid after the call.
template <int NV>
__device__ __forceinline__ void block_sum_staged(const double (&v)[NV], double* sh, double* out)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k * kPNT + threadIdx.x] = v[k];
    __syncthreads();
    for (int k = warp; k < NV; k += kPNT / 32) {
        const double* col = sh + k * kPNT + lane;
        double a = col[0];
#pragma unroll
        for (int i = 1; i < kPNT / 32; ++i) a += col[32 * i];
        a = warp_sum(a);
        if (lane == 0) out[k] = a;
    }
    __syncthreads();
}

static_assert(sizeof(TileSm) >= sizeof(double) * kPNT * kMaxMom, "staging area of the block sums");

// thread 0's state of the device-wide barriers
struct Sync0 {
    unsigned long long base[2];
    unsigned int gen;
};

// Device-wide barrier for thread 0 that sums q (fixed point, unit u); none in
// one-block launches.
__device__ __forceinline__ bool grid_barrier(const AdjP& P, Sync0& y, long long q, double u, double& total)
{
    const int p = (int)(y.gen & 1u);
    y.gen += 1u;
    if (gridDim.x == 1) {
        total = (double)q * u;
        return true;
    }
    return barrier_sum(P.acc + p * kAccStride, y.base[p], q, u, gridDim.x, P.wait_limit, total);
}

// Sum of NV block partials of the barrier with parity p, in block order
// (warp 0; every lane returns the sums).
template <int NV>
__device__ __forceinline__ void sum_partials(const AdjP& P, const BlockSm& B, int p, double (&v)[NV])
{
    const int G = gridDim.x, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0.0;
    if (G == 1) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = B.psum[k];
        return;
    }
    for (int b = lane; b < G; b += 32) {
        const double* pp = P.part + ((size_t)p * G + b) * 4;
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __ldcg(pp + k);
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
}

// copy a Scal from global memory written by other blocks (bypassing L1)
__device__ __forceinline__ void load_scal(Scal& dst, const Scal* src, int tid, int nthr)
{
    static_assert(sizeof(Scal) % 8 == 0, "Scal is copied in 8-byte words");
    const unsigned long long* a = reinterpret_cast<const unsigned long long*>(src);
    unsigned long long* d = reinterpret_cast<unsigned long long*>(&dst);
    for (int k = tid; k < (int)(sizeof(Scal) / 8); k += nthr) d[k] = __ldcg(a + k);
}

__device__ __forceinline__ void load_scal_sm(Scal& dst, const Scal& src, int tid, int nthr)
{
    const unsigned long long* a = reinterpret_cast<const unsigned long long*>(&src);
    unsigned long long* d = reinterpret_cast<unsigned long long*>(&dst);
    for (int k = tid; k < (int)(sizeof(Scal) / 8); k += nthr) d[k] = a[k];
}

// ---- out-of-line closure paths -------------------------------------------------
// The learned closure's code is large and only runs with PBE_KINETICS_MLP; out
// of line it stays out of the instruction stream of the power-law chains.
static __device__ __noinline__ void mlp_backward_64(const Kin& K, const float* x, const double* lo, double* dW,
                                                    float* sm, float* lx)
{
    const float xx[3] = {x[0], x[1], x[2]};
    mlp_backward_block64(K, xx, lo, dW, sm, lx, Bar64());
}

static __device__ __noinline__ StageCoef close1_mlp(Scal* S, const Kin& K, const Geom& g, double V1, double M1,
                                                    const KinT* tpre)
{
    finish_stage1_warp(S, K, V1, M1, tpre);
    return stage_coef_fast<2>(*S, g);
}

static __device__ __noinline__ StageCoef close2_mlp(Scal* S, const Kin& K, const Geom& g, const double* t_out,
                                                    double* rows, const double* mom, int nmom, int vidx,
                                                    const KinT* tpre)
{
    finish_stage2_warp(S, K, g, t_out, rows, mom, nmom, vidx, tpre);
    return stage_coef_fast<1>(*S, g);
}

// One closure evaluation for the weight-gradient kernel: its inputs and the
// adjoints of its outputs (thread 0 of block 0, after the input adjoint).
__device__ __forceinline__ void record_mlp_row(const AdjP& P, BlockSm& B, const float* x)
{
    if (!P.mrows || blockIdx.x != 0 || threadIdx.x != 0) return;
    if (B.nrow < P.mrows_cap) {
        float* r = P.mrows + (size_t)B.nrow * 6;
        r[0] = x[0]; r[1] = x[1]; r[2] = x[2];
        r[3] = (float)B.mlp_lo[0]; r[4] = (float)B.mlp_lo[1]; r[5] = (float)B.mlp_lo[2];
    }
    B.nrow += 1;
}

// ---- adjoint scalar chain ----------------------------------------------------

// Before the stage-2 adjoint of a step (thread 0): seeds of the row the step
// emitted, then the adjoint of C' = C - kappa (V(n') - V(n)) (Eq. 4).
// The chain functions work on a register copy of the adjoint scalars and
// store it back at the end (their updates are dependent, and a shared-memory
// round trip each would lengthen the chain).
__device__ __forceinline__ void rev_begin(const AdjP& P, BlockSm& B, int vidx)
{
    RevS& R = B.R;
    double lC = R.lC;
    if (B.sA.clipped) {
        const double* sd = P.seeds + (size_t)B.sA.out_idx * P.ncol;
        for (int k = 0; k < P.ncol - 2; ++k) R.pc[k] += sd[1 + k];
        lC += sd[P.ncol - 1];
    }
    R.lC = lC;
    R.lV0 = P.K.kappa * lC;
    R.lCprev = lC;
    R.pc[vidx] -= P.K.kappa * lC;
}

// After the stage-2 adjoint (threads 0..63): the step length's share and the
// stage-2 kinetics at (C1, t') (power law or closure backward), then the
// adjoint of C1 = C - kappa (V(n1) - V(n)).
template <int NDIM>
__device__ __forceinline__ void rev_mid(const AdjP& P, BlockSm& B)
{
    constexpr int VIDX = NDIM == 1 ? 3 : 8;
    const Kin& K = P.K;
    const double inv_dA = B.inv_dA;
    const Scal& A = B.sA;
    const Scal& Q = B.sB;
    RevS& R = B.R;
    const double P1 = R.sum[0], P2 = R.sum[1], P0 = R.sum[2], dt = A.dt;
    const double lB = dt * P0 * inv_dA;
    const bool net = K.kind == PBE_KINETICS_MLP && !Q.fbb;   // else the power law (or the closure's fallback)
    if (net) {
        if (threadIdx.x == 0) {
            B.mlp_lo[0] = dt * P1 * Q.G1b;
            B.mlp_lo[1] = NDIM == 2 ? dt * P2 * Q.G2b : 0.0;
            B.mlp_lo[2] = lB * Q.Bb;
            B.run_mlp = Q.G1b > 0.0 || Q.Bb > 0.0;
        }
        Bar64()();
        if (B.run_mlp) {
            float x[3];
            mlp_inputs(K, Q.C1, A.t_new, Q.V1 / Q.M1, x);
            mlp_backward_64(K, x, B.mlp_lo, blockIdx.x == 0 && !P.mrows ? P.dW : nullptr, B.mlp_sm, B.mlp_lx);
            record_mlp_row(P, B, x);
        }
    }
    if (threadIdx.x != 0) return;
    double lth[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) lth[k] = R.lth[k];
    const double ldt = Q.G1b * P1 + Q.G2b * P2 + Q.Bb * P0 * inv_dA;
    double lC1 = 0.0, ltn = R.lt, pv = 0.0, p0 = 0.0;
    if (net) {
        if (B.run_mlp) {
            double lr = 0.0;
            mlp_input_adjoint(K, Q.C1, A.t_new, B.mlp_lx, &lC1, &ltn, &lr);
            pv += lr / Q.M1;
            p0 += -lr * Q.V1 / (Q.M1 * Q.M1);
        }
    } else {
        kin_backward(K, B.ik, Q.C1, A.t_new, Q.G1b, Q.G2b, Q.Bb, Q.Lb, Q.sGb1, Q.sGb2, dt * P1, dt * P2, lB, &lC1,
                     &ltn, lth);
        R.plG1 = dt * P1;
        R.plG2 = dt * P2;
        R.ps = Q.spb;
        R.pL = Q.Lb;
    }
    const double lCprev = R.lCprev, lV0 = R.lV0;
    R.ldt = ldt;
    R.ltn = ltn;
    R.lCprev = lCprev + lC1;
    R.lV0 = lV0 + K.kappa * lC1;
    R.pv = pv - K.kappa * lC1;
    R.p0 = p0;
#pragma unroll
    for (int k = 0; k < 6; ++k) R.lth[k] = lth[k];
    (void)VIDX;
}

// After the stage-1 adjoint (threads 0..63): the step length (CFL branch
// dt = cfl / (G1/dL1 + G2/dL2), or the output clip), the stage-1 kinetics at
// (C, t), and the pending terms of lam for the previous step.
template <int NDIM>
__device__ __forceinline__ void rev_end(const AdjP& P, BlockSm& B)
{
    constexpr int VIDX = NDIM == 1 ? 3 : 8;
    const Kin& K = P.K;
    const Geom& g = P.g;
    const double inv_dA = B.inv_dA;
    const Scal& A = B.sA;
    RevS& R = B.R;
    const double P1 = R.sum[0], P2 = R.sum[1], P0 = R.sum[2], dt = A.dt;
    double ldt = R.ldt + A.G1a * P1 + A.G2a * P2 + A.Ba * P0 * inv_dA;
    double lG1 = dt * P1, lG2 = dt * P2;
    const double lB = dt * P0 * inv_dA;
    if (!A.clipped) {
        ldt += R.ltn;   // t' = t + dt
        const double dR = -(dt * dt) * B.inv_cfl * ldt;   // d(cfl / R)/dR = -dt^2 / cfl
        lG1 += dR * g.inv_d1;
        if (NDIM == 2) lG2 += dR * g.inv_d2;
    }
    const bool net = K.kind == PBE_KINETICS_MLP && !A.fba;   // else the power law (or the closure's fallback)
    if (net) {
        if (threadIdx.x == 0) {
            B.mlp_lo[0] = lG1 * A.G1a;
            B.mlp_lo[1] = NDIM == 2 ? lG2 * A.G2a : 0.0;
            B.mlp_lo[2] = lB * A.Ba;
            B.run_mlp = A.G1a > 0.0 || A.Ba > 0.0;
        }
        Bar64()();
        if (B.run_mlp) {
            float x[3];
            mlp_inputs(K, A.C, A.t, A.V0 / A.M0, x);
            mlp_backward_64(K, x, B.mlp_lo, blockIdx.x == 0 && !P.mrows ? P.dW : nullptr, B.mlp_sm, B.mlp_lx);
            record_mlp_row(P, B, x);
        }
    }
    if (threadIdx.x != 0) return;
    double lth[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) lth[k] = R.lth[k];
    double ltp = A.clipped ? -ldt : R.ltn;   // clipped: dt = t_next - t
    double lC = R.lCprev, pv = 0.0, p0 = 0.0;
    if (net) {
        if (B.run_mlp) {
            double lr = 0.0;
            mlp_input_adjoint(K, A.C, A.t, B.mlp_lx, &lC, &ltp, &lr);
            pv += lr / A.M0;
            p0 += -lr * A.V0 / (A.M0 * A.M0);
        }
    } else {
        kin_backward(K, B.ik, A.C, A.t, A.G1a, A.G2a, A.Ba, A.La, A.sGa1, A.sGa2, lG1, lG2, lB, &lC, &ltp, lth);
        R.plG1 = lG1;
        R.plG2 = lG2;
        R.ps = A.spa;
        R.pL = A.La;
    }
    const double lV0 = R.lV0;
#pragma unroll
    for (int k = 0; k < kMaxMom; ++k) R.pc[k] = 0.0;
    R.pc[VIDX] = pv + lV0;
    R.pc[0] += p0;
    R.lC = lC;
    R.lt = ltp;
#pragma unroll
    for (int k = 0; k < 6; ++k) R.lth[k] = lth[k];
}

// ---- forward step --------------------------------------------------------------
// One SSP-RK2 step with its scalar chains, every block on its own tiles:
// stage 1 in1 -> n1, the device-wide barrier with the volume moment (and mu0
// for the closure), the stage-1 close and the stage-2 kinetics; stage 2 ->
// out2, the barrier, the step close and the next step's kinetics and length.
// With q >= 0 block 0 records the scalars (recA[q] at the start, recB[q]
// after the stage-1 close).  emit: the
// forward pass (output rows and their per-block moments); with stage2 false
// (the last step of a recomputed segment) only stage 1 and its close run.
// Returns false when a device-wide wait ran out.
template <int NDIM>
__device__ __forceinline__ bool fwd_step(const AdjP& P, BlockSm& B, Sync0& y, const double* in1, double* n1,
                                         double* out2, int q, bool emit, bool stage2, int t_first, int t_end,
                                         double u, double inv_u)
{
    constexpr int NM = NDIM == 1 ? 4 : 10;
    constexpr int VIDX = NDIM == 1 ? 3 : 8;
    const bool mlp = P.K.kind == PBE_KINETICS_MLP;
    const int warp = threadIdx.x >> 5;
    const int G = gridDim.x;
    // temperature and solubility at the step's end, where both kinetics of the step are evaluated
    KinT tpre{0.0, 0.0};
    if (warp == 0 && P.K.kind != PBE_KINETICS_FIXED) tpre = kin_temperature(P.K, B.s.t_new);
    if (q >= 0 && threadIdx.x == 0 && blockIdx.x == 0) P.recA[q] = B.s;
#pragma unroll 1
    for (int stage = 1; stage <= 2; ++stage) {
        if (stage == 2 && B.s.done) break;   // the stage-1 close failed (non-finite)
        const StageCoef sc = B.sc;
        const bool moms = emit && stage == 2 && sc.moms;
        double m[kMaxMom];
#pragma unroll
        for (int k = 0; k < kMaxMom; ++k) m[k] = 0.0;
        for (int t = t_first; t < t_end; ++t) {
            int i0, j0;
            tile_org<NDIM>(P, t, i0, j0);
            if constexpr (NDIM == 1) {
                if (stage == 1) fwd_tile1d<1>(in1, nullptr, n1, i0, P.t1, P.g, sc, false, mlp, m, B.t.f1);
                else fwd_tile1d<2>(n1, in1, out2, i0, P.t1, P.g, sc, moms, mlp, m, B.t.f1);
            } else {
                if (stage == 1) fwd_tile2d<1>(in1, nullptr, n1, i0, j0, P.ti, P.g, sc, false, mlp, m, B.t.f2);
                else fwd_tile2d<2>(n1, in1, out2, i0, j0, P.ti, P.g, sc, moms, mlp, m, B.t.f2);
            }
        }
        const long long qb = block_sum_fixed_t0(m[VIDX], inv_u, B.wsum);
        const int parity = (int)(y.gen & 1u);   // meaningful in thread 0
        if (moms || mlp) {
            double mm[NM];
#pragma unroll
            for (int k = 0; k < NM; ++k) mm[k] = m[k];
            block_sum_staged<NM>(mm, reinterpret_cast<double*>(&B.t), B.red);
            if (threadIdx.x == 0) {
                if (moms)
                    for (int k = 0; k < NM; ++k) P.rowpart[((size_t)B.s.out_idx * G + blockIdx.x) * NM + k] = B.red[k];
                if (mlp) {
                    B.psum[0] = B.red[0];
                    P.part[((size_t)parity * G + blockIdx.x) * 4] = B.red[0];
                }
            }
        }
        if (threadIdx.x == 0) {
            double tot = 0.0;
            B.fail = !grid_barrier(P, y, qb, u, tot);
            B.vtot = tot;
            B.par = parity;
        }
        __syncthreads();
        if (B.fail) return false;
        if (warp == 0) {
            double M = 1.0;
            if (mlp) {
                double v[1];
                sum_partials<1>(P, B, B.par, v);
                M = v[0];
            }
            StageCoef nx;
            if (stage == 1) {
                if (mlp) {
                    nx = close1_mlp(&B.s, P.K, P.g, B.vtot, M, &tpre);
                } else {
                    nx = fused_finish1(&B.s, P.K, P.g, B.vtot, tpre);
                }
                if (q >= 0 && threadIdx.x == 0 && blockIdx.x == 0) P.recB[q] = B.s;
            } else {
                double mom[kMaxMom];
#pragma unroll
                for (int k = 0; k < kMaxMom; ++k) mom[k] = 0.0;
                mom[0] = M;
                mom[VIDX] = B.vtot;
                double* rows = emit && blockIdx.x == 0 ? P.rows : nullptr;
                if (mlp) {
                    nx = close2_mlp(&B.s, P.K, P.g, P.t_out, rows, mom, NM, VIDX, &tpre);
                } else {
                    nx = fused_finish2(&B.s, P.K, P.g, P.t_out, rows, mom, NM, VIDX, tpre);
                }
            }
            if (threadIdx.x == 0) B.sc = nx;
        }
        __syncthreads();
        if (!stage2) break;
    }
    return true;
}

// dL/da_mk += dL/dG_m s^k for the stage just reversed (warp 0 of block 0; lane
// l owns the terms k0 .. k0 + c - 1 as in poly_growth_warp, so the sums keep
// a fixed order).  Nothing when S <= 1 (s = 0: the rates were 0).
__device__ __forceinline__ void poly_grad_accumulate(const Kin& K, const RevS& R, double* dpoly)
{
    const double s = R.ps;
    if (!(s > 0.0)) return;
    const int lane = threadIdx.x & 31, n = K.npoly;
    const int c = (n + 31) >> 5, k0 = lane * c + 1;
    if (k0 > n) return;
    const int k1 = min(n, k0 + c - 1);
    const double lG[2] = {R.plG1, R.plG2};
    double sk = k0 == 1 ? s : pbe_exp_tab((double)k0 * R.pL);
    for (int k = k0; k <= k1; ++k) {
        for (int m = 0; m < K.ndim; ++m) dpoly[(size_t)m * n + k - 1] += lG[m] * sk;
        sk *= s;
    }
}

// ---- the kernel ------------------------------------------------------------------
template <int NDIM>
__global__ void __launch_bounds__(kPNT, 1) k_adjoint_persistent(AdjP P)
{
    constexpr int NM = NDIM == 1 ? 4 : 10;
    constexpr int VIDX = NDIM == 1 ? 3 : 8;
    __shared__ BlockSm B;
    const int G = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t_first = (int)(((long long)blockIdx.x * P.ntiles) / G);
    const int t_end = (int)(((long long)(blockIdx.x + 1) * P.ntiles) / G);
    Sync0 y;
    y.base[0] = y.base[1] = 0ull;
    y.gen = 0u;
    if (threadIdx.x == 0) {
        B.s = *P.S;
        B.sc = stage_coef_fast<1>(B.s, P.g);
        B.fail = 0;
        B.ik[0] = P.K.kg1 > 0.0 ? 1.0 / P.K.kg1 : 0.0;
        B.ik[1] = P.K.kg2 > 0.0 ? 1.0 / P.K.kg2 : 0.0;
        B.ik[2] = P.K.kb > 0.0 ? 1.0 / P.K.kb : 0.0;
        B.inv_dA = NDIM == 1 ? P.g.inv_d1 : P.g.inv_d1 * P.g.inv_d2;
        B.nrow = 0;
        B.inv_cfl = 1.0 / P.K.cfl;
        memset(&B.R, 0, sizeof(RevS));
    }
    __syncthreads();
    const int row_first = B.s.out_idx;   // rows before it came from the prologue
    // unit of the fixed-point volume sums (as in the fused solve): 2^(E-52)
    // with 2^E above twice the largest volume moment the solute balance allows
    double u, inv_u;
    {
        double vmax = 2.0 * (B.s.V0 + (P.K.kappa > 0.0 ? B.s.C / P.K.kappa : 0.0));
        if (!(vmax > 0.0) || !isfinite(vmax)) vmax = 1.0;
        const int E = ilogb(vmax) + 1;
        u = ldexp(1.0, E - 52);
        inv_u = ldexp(1.0, 52 - E);
    }
    int status = PBE_OK;
    if (P.fwd_only) {
        // ---- a solve only (the fused path's closure solves): the state alternates
        // between n and fin, the stage-1 output goes to u, nothing is recorded ----
        double* cur = P.n;
        double* nxt = P.fin;
        while (!B.s.done) {
            if (!fwd_step<NDIM>(P, B, y, cur, P.u, nxt, -1, true, true, t_first, t_end, u, inv_u)) {
                status = PBE_ETIMEOUT;
                break;
            }
            if (!B.s.done || B.s.status == PBE_OK) {
                double* tmp = cur;
                cur = nxt;
                nxt = tmp;
            }
        }
        if (status == PBE_OK && B.s.status != PBE_OK) status = B.s.status;
        if (status == PBE_OK && cur != P.n) {   // the final state into n (own cells: no barrier needed)
            for (int t = t_first; t < t_end; ++t) {
                int i0, j0;
                tile_org<NDIM>(P, t, i0, j0);
                const int rows_t = NDIM == 1 ? 1 : P.ti, cols_t = NDIM == 1 ? P.t1 : kPTJ;
                for (int k = threadIdx.x; k < rows_t * cols_t; k += kPNT) {
                    const int i = i0 + (NDIM == 1 ? k : k / cols_t), j = j0 + (NDIM == 1 ? 0 : k % cols_t);
                    if (i < P.g.N1 && j < P.g.N2) {
                        const size_t gi = (size_t)i * P.g.N2 + j;
                        P.n[gi] = __ldcg(cur + gi);
                    }
                }
            }
        }
        if (threadIdx.x == 0 && status == PBE_ETIMEOUT) {   // every block that gave up marks the solve
            P.S->status = PBE_ETIMEOUT;
            P.S->done = 1;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (status != PBE_ETIMEOUT) {
                B.s.counter = 0u;
                *P.S = B.s;
            }
            P.out->status = status;
            P.out->steps = B.s.steps;
            P.out->row_first = row_first;
            P.out->row_end = B.s.out_idx;
        }
        return;
    }
    // ---- forward pass ----
    int c = 0, q = 0;
    while (!B.s.done) {
        if (q == 0) {
            if (c >= P.ck_cap) { status = kStatusGrow; break; }
            if (threadIdx.x == 0 && blockIdx.x == 0) P.ckS[c] = B.s;
        }
        double* out2 = q + 1 < P.Kc ? st_ptr(P, c, q + 1) : st_ptr(P, c + 1, 0);
        if (!fwd_step<NDIM>(P, B, y, st_ptr(P, c, q), P.seg_n1 + (size_t)q * P.nc, out2, q, true, true, t_first,
                            t_end, u, inv_u)) {
            status = PBE_ETIMEOUT;
            break;
        }
        if (++q == P.Kc) { q = 0; ++c; }
    }
    if (status == PBE_OK && B.s.status != PBE_OK) status = B.s.status;
    if (status != PBE_OK) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            P.out->status = status;
            P.out->steps = B.s.steps;
            P.out->row_first = row_first;
            P.out->row_end = B.s.out_idx;
        }
        return;
    }
    // keep the final state (its slot may be overwritten by recomputed segments)
    {
        const double* src = st_ptr(P, c, q);
        for (int t = t_first; t < t_end; ++t) {
            int i0, j0;
            tile_org<NDIM>(P, t, i0, j0);
            const int rows_t = NDIM == 1 ? 1 : P.ti, cols_t = NDIM == 1 ? P.t1 : kPTJ;
            for (int k = threadIdx.x; k < rows_t * cols_t; k += kPNT) {
                const int i = i0 + (NDIM == 1 ? k : k / cols_t), j = j0 + (NDIM == 1 ? 0 : k % cols_t);
                if (i < P.g.N1 && j < P.g.N2) {
                    const size_t gi = (size_t)i * P.g.N2 + j;
                    P.fin[gi] = __ldcg(src + gi);
                }
            }
        }
    }
    if (threadIdx.x == 0) B.sfin = B.s;
    __syncthreads();
    // ---- reverse sweep ----
    const long long total = B.sfin.steps;
    const int nseg = (int)((total + P.Kc - 1) / P.Kc);
    double* lam = P.lamA;
    double* lamo = P.lamB;
    const double dA = NDIM == 1 ? P.g.d1 : P.g.d1 * P.g.d2;
    for (int cc = nseg - 1; cc >= 0 && status == PBE_OK; --cc) {
        const int len = (int)min((long long)P.Kc, total - (long long)cc * P.Kc);
        if (cc < nseg - 1) {   // recompute the segment from its checkpoint
            if (warp == 0) load_scal(B.s, P.ckS + cc, lane, 32);
            __syncthreads();
            if (threadIdx.x == 0) B.sc = stage_coef_fast<1>(B.s, P.g);
            __syncthreads();
            for (int qq = 0; qq < len; ++qq)
                if (!fwd_step<NDIM>(P, B, y, st_ptr(P, cc, qq), P.seg_n1 + (size_t)qq * P.nc,
                                    qq + 1 < len ? st_ptr(P, cc, qq + 1) : nullptr, qq, false, qq + 1 < len,
                                    t_first, t_end, u, inv_u)) {
                    status = PBE_ETIMEOUT;
                    break;
                }
            if (status != PBE_OK) break;
            // the last recomputed step ran stage 1 only, and block 0 recorded its
            // stage-1 close after that stage's barrier: one more barrier makes the
            // record visible to every block before the reverse sweep reads it
            if (threadIdx.x == 0) {
                double unused;
                B.fail = !grid_barrier(P, y, 0, u, unused);
            }
            __syncthreads();
            if (B.fail) { status = PBE_ETIMEOUT; break; }
        }
        for (int qq = len - 1; qq >= 0; --qq) {
            if (warp == 0) {
                if (qq == len - 1) {
                    load_scal(B.sA, P.recA + qq, lane, 32);
                    load_scal(B.sB, P.recB + qq, lane, 32);
                } else {   // prefetched during the previous step
                    load_scal_sm(B.sA, B.nA, lane, 32);
                    load_scal_sm(B.sB, B.nB, lane, 32);
                }
                __syncwarp();
                if (lane == 0) rev_begin(P, B, VIDX);
            }
            __syncthreads();
#pragma unroll 1
            for (int stage = 2; stage >= 1; --stage) {
                double acc[3] = {0.0, 0.0, 0.0};
                const double dt = B.sA.dt;
                // the next step's records: loads issued now, stored after the cells
                unsigned long long pre[2] = {0ull, 0ull};
                const bool prefetch = stage == 2 && qq > 0 && warp == 0 && lane < (int)(sizeof(Scal) / 8);
                if (prefetch) {
                    pre[0] = __ldcg(reinterpret_cast<const unsigned long long*>(P.recA + qq - 1) + lane);
                    pre[1] = __ldcg(reinterpret_cast<const unsigned long long*>(P.recB + qq - 1) + lane);
                }
                double* own = (t_end - t_first == 1) ? B.own : nullptr;
                for (int t = t_first; t < t_end; ++t) {
                    int i0, j0;
                    tile_org<NDIM>(P, t, i0, j0);
                    if constexpr (NDIM == 1) {
                        if (stage == 2)
                            rev_tile1d<2>(P.seg_n1 + (size_t)qq * P.nc, lam, lamo, P.u, i0, P.t1, P.g, dt, B.sB.G1b, B.R,
                                          acc, own, B.t.r1);
                        else
                            rev_tile1d<1>(st_ptr(P, cc, qq), P.u, lamo, nullptr, i0, P.t1, P.g, dt, B.sA.G1a, B.R, acc,
                                          own, B.t.r1);
                    } else {
                        if (stage == 2)
                            rev_tile2d<2>(P.seg_n1 + (size_t)qq * P.nc, lam, lamo, P.u, i0, j0, P.ti, P.g, dt, B.sB.G1b,
                                          B.sB.G2b, B.R, acc, own, B.t.r2);
                        else
                            rev_tile2d<1>(st_ptr(P, cc, qq), P.u, lamo, nullptr, i0, j0, P.ti, P.g, dt, B.sA.G1a,
                                          B.sA.G2a, B.R, acc, own, B.t.r2);
                    }
                }
                if (prefetch) {
                    reinterpret_cast<unsigned long long*>(&B.nA)[lane] = pre[0];
                    reinterpret_cast<unsigned long long*>(&B.nB)[lane] = pre[1];
                }
                block_sum_staged<3>(acc, reinterpret_cast<double*>(&B.t), B.red);
                if (threadIdx.x == 0) {
                    const int parity = (int)(y.gen & 1u);
                    B.par = parity;
                    for (int k = 0; k < 3; ++k) B.psum[k] = B.red[k];
                    if (G > 1)
                        for (int k = 0; k < 3; ++k) P.part[((size_t)parity * G + blockIdx.x) * 4 + k] = B.red[k];
                    double dummy;
                    B.fail = !grid_barrier(P, y, 0, u, dummy);
                }
                __syncthreads();
                if (B.fail) { status = PBE_ETIMEOUT; break; }
                if (warp == 0) {
                    double v[3];
                    sum_partials<3>(P, B, B.par, v);
                    if (lane == 0) { B.R.sum[0] = v[0]; B.R.sum[1] = v[1]; B.R.sum[2] = v[2]; }
                    __syncwarp();
                }
                if (threadIdx.x < 64) {
                    if (stage == 2) rev_mid<NDIM>(P, B);
                    else rev_end<NDIM>(P, B);
                }
                __syncthreads();
                if (P.K.growth_form == 2 && blockIdx.x == 0 && warp == 0) poly_grad_accumulate(P.K, B.R, P.dpoly);
            }
            if (status != PBE_OK) break;
            double* tmp = lam;
            lam = lamo;
            lamo = tmp;
        }
    }
    if (status != PBE_OK) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            P.out->status = status;
            P.out->steps = total;
            P.out->row_first = row_first;
            P.out->row_end = B.sfin.out_idx;
        }
        return;
    }
    // seeds of a row emitted at the start time, then lam0 = lam + pending terms into lamA
    if (threadIdx.x == 0 && P.t_out[0] == P.t0) {
        for (int k = 0; k < P.ncol - 2; ++k) B.R.pc[k] += P.seeds[1 + k];
        B.R.lC += P.seeds[P.ncol - 1];
    }
    __syncthreads();
    for (int t = t_first; t < t_end; ++t) {
        int i0, j0;
        tile_org<NDIM>(P, t, i0, j0);
        const int rows_t = NDIM == 1 ? 1 : P.ti, cols_t = NDIM == 1 ? P.t1 : kPTJ;
        for (int k = threadIdx.x; k < rows_t * cols_t; k += kPNT) {
            const int i = i0 + (NDIM == 1 ? k : k / cols_t), j = j0 + (NDIM == 1 ? 0 : k % cols_t);
            if (i < P.g.N1 && j < P.g.N2) {
                const size_t gi = (size_t)i * P.g.N2 + j;
                P.lamA[gi] = __ldcg(lam + gi) + poly_weights<NDIM>(B.R.pc, (i + 0.5) * P.g.d1, (j + 0.5) * P.g.d2, dA);
                P.n[gi] = P.fin[gi];
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        B.sfin.counter = 0u;
        *P.S = B.sfin;
        for (int k = 0; k < 6; ++k) P.out->lth[k] = B.R.lth[k];
        P.out->lC = B.R.lC;
        P.out->steps = total;
        P.out->nrows = B.nrow;
        P.out->status = PBE_OK;
        P.out->row_first = row_first;
        P.out->row_end = B.sfin.out_idx;
    }
    (void)NM;
}

// Moments of the rows the forward pass emitted: sums of the per-block
// partials in block order (one block per row, one warp per moment).
template <int NDIM>
__global__ void k_adjoint_rows(const double* rowpart, int G, const AdjOut* out, double* rows)
{
    constexpr int NM = NDIM == 1 ? 4 : 10;
    const int r = out->row_first + blockIdx.x;
    const int m = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (r >= out->row_end || m >= NM) return;
    double acc = 0.0;
    for (int b = lane; b < G; b += 32) acc += rowpart[((size_t)r * G + b) * NM + m];
    acc = warp_sum(acc);
    if (lane == 0) rows[(size_t)r * (NM + 2) + 1 + m] = acc;
}

}  // namespace pbe

// ---- host side ---------------------------------------------------------------------
void pbe_set_error_message(int code, const char* msg);  // pbe_api.cu

namespace pbe {

struct AdjWork {
    int K, ck_cap, seeds_cap;
    int G, ntiles, tiles_x, ti, t1;
    long long last_total;   // steps of the last gradient (sizes the checkpoint store of the next)
    double *seg_n, *seg_n1, *ck, *lamA, *lamB, *u, *part, *seeds, *dW;
    double* dpoly;          // dL/d(growth polynomial coefficients) of the last gradient
    int dpoly_cap;
    float* mrows;           // closure rows of the last gradient (6 floats each)
    long long mrows_cap, last_nrows;   // capacity; rows of the last fused-path gradient (-1: none)
    float* gpart;           // workspace of the weight-gradient kernel
    float* catrows;         // rows of several grids side by side (pbe_closure_grad)
    long long catrows_cap;
    Scal *recA, *recB, *ckS;
    AdjOut* out;
    AdjOut* h_out;          // pinned
};

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

#define PTRY(call)                                                                                        \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return afail(PBE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

template <class T>
cudaError_t grow(T** p, size_t count)
{
    cudaFree(*p);
    *p = nullptr;
    return cudaMalloc(p, sizeof(T) * (count ? count : 1));
}

// Blocks and tiles of the launch: 2-D tiles of ti x 32 cells with the
// smallest ti (>= 4) that gives every SM at most one tile, up to 16 rows
// (larger grids: 16-row tiles, several a block); 1-D tiles of 64..512 cells
// chosen the same way.
cudaError_t adjoint_config(pbe_grid* g, AdjWork* w)
{
    if (w->G) return cudaSuccess;
    const void* fn = g->geo.ndim == 1 ? (const void*)k_adjoint_persistent<1> : (const void*)k_adjoint_persistent<2>;
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kPNT, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int cap = std::min(g->sms * occ, g->max_blocks / 2);
    cap = std::min(cap, 1000);   // the arrival count of barrier_sum has 10 bits
    if (g->block_limit > 0) cap = std::min(cap, g->block_limit);
    if (g->geo.ndim == 1) {
        // tiles of a multiple of 32 cells, at least kPT1Min, that give every block at most one when the grid allows
        const int nb = std::min(g->sms, cap);
        const int per = (g->geo.N1 + nb - 1) / nb;
        w->t1 = std::min(kPT1, std::max(kPT1Min, (per + 31) / 32 * 32));
        w->tiles_x = 1;
        w->ti = 1;
        w->ntiles = (g->geo.N1 + w->t1 - 1) / w->t1;
    } else {
        w->tiles_x = (g->geo.N2 + kPTJ - 1) / kPTJ;
        const int per = std::max(1, std::min(g->sms, cap) / w->tiles_x);
        int ti = (g->geo.N1 + per - 1) / per;
        w->ti = std::min(kPTI, std::max(4, ti));
        w->ntiles = w->tiles_x * ((g->geo.N1 + w->ti - 1) / w->ti);
    }
    w->G = std::max(1, std::min(w->ntiles, cap));
    return cudaSuccess;
}

}  // namespace

void adjoint_work_free(pbe_grid* g)
{
    AdjWork* w = g->adjw;
    if (!w) return;
    cudaFree(w->seg_n); cudaFree(w->seg_n1); cudaFree(w->ck); cudaFree(w->lamA); cudaFree(w->lamB);
    cudaFree(w->u); cudaFree(w->part); cudaFree(w->seeds); cudaFree(w->dW); cudaFree(w->dpoly);
    cudaFree(w->mrows); cudaFree(w->gpart); cudaFree(w->catrows);
    cudaFree(w->recA); cudaFree(w->recB); cudaFree(w->ckS); cudaFree(w->out);
    cudaFreeHost(w->h_out);
    delete w;
    g->adjw = nullptr;
}

// A solve of the fused path with the learned closure: the persistent kernel's
// forward pass alone (its per-stage mu0 sums give the closure's moment-ratio
// input).  The caller has put the output times on the device; like the fused
// solve it leaves the rows in d_rows and the scalars in d_S and does not
// synchronize.
cudaError_t launch_solve_persistent(pbe_grid* g, int n_out)
{
    if (!g->adjw) {
        g->adjw = new AdjWork();
        memset((void*)g->adjw, 0, sizeof(AdjWork));
        cudaError_t e = cudaMallocHost(&g->adjw->h_out, sizeof(AdjOut));
        if (e != cudaSuccess) return e;
    }
    AdjWork* w = g->adjw;
    cudaError_t e = adjoint_config(g, w);
    if (e != cudaSuccess) return e;
    const size_t nc = g->ncell;
    cudaStream_t st = g->stream;
    if (!w->u || !w->part || !w->out) {
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        if ((e = grow(&w->u, nc)) != cudaSuccess || (e = grow(&w->part, (size_t)2 * w->G * 4)) != cudaSuccess ||
            (e = grow(&w->out, (size_t)1)) != cudaSuccess)
            return e;
    }
    if ((e = cudaMemsetAsync(g->d_bar, 0, 2 * kAccStride * sizeof(unsigned long long), st)) != cudaSuccess) return e;
    AdjP P;
    memset(&P, 0, sizeof(P));
    P.n = g->d_n; P.fin = g->d_n1; P.S = g->d_S; P.K = g->kin; P.g = g->geo;
    P.t_out = g->d_tout; P.rows = g->d_rows; P.rowpart = g->d_rowpart;
    P.u = w->u; P.part = w->part; P.out = w->out;
    P.acc = reinterpret_cast<unsigned long long*>(g->d_bar);
    P.nc = nc; P.Kc = 1; P.n_out = n_out; P.ncol = g->geo.ndim == 1 ? 6 : 12;
    P.ntiles = w->ntiles; P.tiles_x = w->tiles_x; P.ti = w->ti; P.t1 = w->t1;
    P.wait_limit = g->wait_cycles > 0 ? g->wait_cycles : (g->wait_cycles == 0 ? 0 : kBarrierCycles);
    P.fwd_only = 1;
    void* args[] = {&P};
    const void* fn = g->geo.ndim == 1 ? (const void*)k_adjoint_persistent<1> : (const void*)k_adjoint_persistent<2>;
    if (g->timing && (e = cudaEventRecord(g->ev_k0, st)) != cudaSuccess) return e;
    if ((e = cudaLaunchCooperativeKernel(fn, w->G, kPNT, args, 0, st)) != cudaSuccess) return e;
    if (g->timing && (e = cudaEventRecord(g->ev_k1, st)) != cudaSuccess) return e;
    const int nm = g->geo.ndim == 1 ? 4 : 10;
    if (g->geo.ndim == 1) k_adjoint_rows<1><<<n_out, nm * 32, 0, st>>>(g->d_rowpart, w->G, w->out, g->d_rows);
    else k_adjoint_rows<2><<<n_out, nm * 32, 0, st>>>(g->d_rowpart, w->G, w->out, g->d_rows);
    return cudaGetLastError();
}

pbe_status vjp_persistent(pbe_grid* g, const double* t_out, int n_out, const double* seeds_in, int seeds_mem, int K,
                          double* dL_dtheta, double* dL_dn0, double* dL_dC0, double* rows, int mem,
                          double* dL_dweights)
{
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != g->device) PTRY(cudaSetDevice(g->device));
    struct Restore {
        int dev;
        ~Restore() { if (dev >= 0) cudaSetDevice(dev); }
    } restore{prev != g->device ? prev : -1};
    cudaStream_t st = g->stream;
    const size_t nc = g->ncell;
    const int ndim = g->geo.ndim, ncol = ndim == 1 ? 6 : 12, nm = ndim == 1 ? 4 : 10;
    pbe_status ps = prepare_tout(g, t_out, n_out);
    if (ps != PBE_OK) return ps;
    if (!g->adjw) {
        g->adjw = new AdjWork();
        memset((void*)g->adjw, 0, sizeof(AdjWork));
        PTRY(cudaMallocHost(&g->adjw->h_out, sizeof(AdjOut)));
    }
    AdjWork* w = g->adjw;
    PTRY(adjoint_config(g, w));
    // buffers sized once per grid and grown when a call needs more
    bool realloc_seg = w->K != K, need_ck = false;
    if (realloc_seg || !w->lamA || w->seeds_cap < n_out * ncol) PTRY(cudaStreamSynchronize(st));
    if (realloc_seg) {
        if (grow(&w->seg_n, (size_t)std::max(K - 1, 1) * nc) != cudaSuccess ||
            grow(&w->seg_n1, (size_t)K * nc) != cudaSuccess || grow(&w->recA, (size_t)K) != cudaSuccess ||
            grow(&w->recB, (size_t)K) != cudaSuccess) {
            w->K = 0;
            cudaGetLastError();
            return afail(PBE_ENOMEM, "allocating the adjoint's segment store (%d steps of %zu cells) failed", K, nc);
        }
        w->K = K;
        need_ck = true;
    }
    if (!w->lamA) {
        if (grow(&w->lamA, nc) != cudaSuccess || grow(&w->lamB, nc) != cudaSuccess || grow(&w->u, nc) != cudaSuccess ||
            grow(&w->part, (size_t)2 * w->G * 4) != cudaSuccess || grow(&w->dW, (size_t)kMlpNW) != cudaSuccess ||
            grow(&w->out, (size_t)1) != cudaSuccess) {
            cudaFree(w->lamA);
            w->lamA = nullptr;
            cudaGetLastError();
            return afail(PBE_ENOMEM, "allocating the adjoint work buffers failed");
        }
    }
    if (w->seeds_cap < n_out * ncol) {
        if (grow(&w->seeds, (size_t)n_out * ncol) != cudaSuccess) {
            w->seeds_cap = 0;
            cudaGetLastError();
            return afail(PBE_ENOMEM, "allocating the adjoint seeds failed");
        }
        w->seeds_cap = n_out * ncol;
    }
    // checkpoints: room for twice the steps of the last gradient (or the output count)
    const long long hint = std::max<long long>(w->last_total, n_out);
    int want_ck = (int)std::min<long long>((2 * hint + K - 1) / K + 1, 1 << 20);
    want_ck = std::max(want_ck, 4);
    if (w->ck_cap < want_ck || need_ck) {
        PTRY(cudaStreamSynchronize(st));
        if (grow(&w->ck, (size_t)want_ck * nc) != cudaSuccess || grow(&w->ckS, (size_t)want_ck + 1) != cudaSuccess) {
            w->ck_cap = 0;
            cudaGetLastError();
            return afail(PBE_ENOMEM, "allocating %d adjoint checkpoints of %zu cells failed", want_ck, nc);
        }
        w->ck_cap = want_ck;
    }
    const int npoly_all = g->kin.growth_form == 2 ? g->kin.npoly * ndim : 0;
    if (npoly_all > w->dpoly_cap) {
        PTRY(cudaStreamSynchronize(st));
        if (grow(&w->dpoly, (size_t)npoly_all) != cudaSuccess) {
            w->dpoly_cap = 0;
            cudaGetLastError();
            return afail(PBE_ENOMEM, "allocating the polynomial-coefficient gradient failed");
        }
        w->dpoly_cap = npoly_all;
    }
    const bool mlp = g->kin.kind == PBE_KINETICS_MLP;
    w->last_nrows = -1;
    if (mlp) {
        const long long cap = 2LL * w->ck_cap * K + 2;
        if (w->mrows_cap < cap || !w->gpart) {
            PTRY(cudaStreamSynchronize(st));
            if (grow(&w->mrows, (size_t)cap * 6) != cudaSuccess ||
                (!w->gpart && grow(&w->gpart, (size_t)mlp_grad_part_floats()) != cudaSuccess)) {
                w->mrows_cap = 0;
                cudaGetLastError();
                return afail(PBE_ENOMEM, "allocating the closure's gradient rows failed");
            }
            w->mrows_cap = cap;
        }
    }
    PTRY(cudaMemcpyAsync(w->seeds, seeds_in, sizeof(double) * ncol * n_out,
                         seeds_mem == PBE_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    const long long wait_limit = g->wait_cycles > 0 ? g->wait_cycles : (g->wait_cycles == 0 ? 0 : kBarrierCycles);
    const double t0 = g->t_host;
    g->kernel_ms = -1.0;
    for (int attempt = 0;; ++attempt) {
        PTRY(cudaMemsetAsync(w->lamA, 0, sizeof(double) * nc, st));
        PTRY(cudaMemsetAsync(g->d_bar, 0, 2 * kAccStride * sizeof(unsigned long long), st));
        if (g->kin.kind == PBE_KINETICS_MLP) PTRY(cudaMemsetAsync(w->dW, 0, sizeof(double) * kMlpNW, st));
        if (npoly_all) PTRY(cudaMemsetAsync(w->dpoly, 0, sizeof(double) * npoly_all, st));
        PTRY(launch_prologue(g, n_out, g->max_steps, nullptr));
        AdjP P;
        memset(&P, 0, sizeof(P));
        P.n = g->d_n; P.fin = g->d_n1; P.S = g->d_S; P.K = g->kin; P.g = g->geo;
        P.t_out = g->d_tout; P.rows = g->d_rows; P.rowpart = g->d_rowpart;
        P.seg_n = w->seg_n; P.seg_n1 = w->seg_n1; P.ck = w->ck; P.recA = w->recA; P.recB = w->recB; P.ckS = w->ckS;
        P.lamA = w->lamA; P.lamB = w->lamB; P.u = w->u; P.part = w->part; P.seeds = w->seeds; P.dW = w->dW;
        P.dpoly = w->dpoly;
        P.mrows = mlp ? w->mrows : nullptr;
        P.mrows_cap = mlp ? w->mrows_cap : 0;
        P.out = w->out; P.acc = reinterpret_cast<unsigned long long*>(g->d_bar);
        P.nc = nc; P.Kc = K; P.ck_cap = w->ck_cap; P.n_out = n_out; P.ncol = ncol;
        P.ntiles = w->ntiles; P.tiles_x = w->tiles_x; P.ti = w->ti; P.t1 = w->t1; P.wait_limit = wait_limit; P.t0 = t0;
        void* args[] = {&P};
        const void* fn = ndim == 1 ? (const void*)k_adjoint_persistent<1> : (const void*)k_adjoint_persistent<2>;
        if (g->timing) PTRY(cudaEventRecord(g->ev_k0, st));
        PTRY(cudaLaunchCooperativeKernel(fn, w->G, kPNT, args, 0, st));
        if (g->timing) PTRY(cudaEventRecord(g->ev_k1, st));
        if (ndim == 1) k_adjoint_rows<1><<<n_out, nm * 32, 0, st>>>(g->d_rowpart, w->G, w->out, g->d_rows);
        else k_adjoint_rows<2><<<n_out, nm * 32, 0, st>>>(g->d_rowpart, w->G, w->out, g->d_rows);
        PTRY(cudaGetLastError());
        PTRY(cudaMemcpyAsync(w->h_out, w->out, sizeof(AdjOut), cudaMemcpyDeviceToHost, st));
        PTRY(cudaMemcpyAsync(g->h_S, g->d_S, sizeof(Scal), cudaMemcpyDeviceToHost, st));
        PTRY(cudaStreamSynchronize(st));
        if (w->h_out->status != kStatusGrow || attempt >= 12) break;
        // the checkpoint store was full: twice as many slots, and run again
        const int cap = w->ck_cap * 2;
        if (grow(&w->ck, (size_t)cap * nc) != cudaSuccess || grow(&w->ckS, (size_t)cap + 1) != cudaSuccess) {
            w->ck_cap = 0;
            cudaGetLastError();
            return afail(PBE_ENOMEM, "allocating %d adjoint checkpoints of %zu cells failed", cap, nc);
        }
        w->ck_cap = cap;
        if (mlp) {   // room for two closure rows a step of the larger store
            const long long rcap = 2LL * cap * K + 2;
            if (grow(&w->mrows, (size_t)rcap * 6) != cudaSuccess) {
                w->mrows_cap = 0;
                cudaGetLastError();
                return afail(PBE_ENOMEM, "allocating the closure's gradient rows failed");
            }
            w->mrows_cap = rcap;
        }
    }
    const AdjOut o = *w->h_out;
    if (o.status == PBE_ENONFINITE) return afail(PBE_ENONFINITE, "non-finite value in the forward pass of the gradient");
    if (o.status == PBE_ETIMEOUT)
        return afail(PBE_ETIMEOUT, "step budget exhausted or a device-wide wait ran out in the gradient");
    if (o.status != PBE_OK) return afail(PBE_ECUDA, "persistent adjoint reported status %d", o.status);
    w->last_total = o.steps;
    if (g->timing) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, g->ev_k0, g->ev_k1) == cudaSuccess) g->kernel_ms = ms;
    }
    if (rows)
        PTRY(cudaMemcpyAsync(rows, g->d_rows, sizeof(double) * ncol * n_out,
                             mem == PBE_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (dL_dn0)
        PTRY(cudaMemcpyAsync(dL_dn0, w->lamA, sizeof(double) * nc,
                             mem == PBE_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (mlp) {
        if (o.nrows > w->mrows_cap) return afail(PBE_ECUDA, "closure rows beyond their store (%lld)", o.nrows);
        w->last_nrows = o.nrows;
        if (dL_dweights) {
            PTRY(launch_mlp_grad(w->mrows, o.nrows, g->d_mW, g->d_mB, w->gpart, w->dW, st));
            PTRY(cudaMemcpyAsync(dL_dweights, w->dW, sizeof(double) * kMlpNW, cudaMemcpyDeviceToHost, st));
        }
    } else if (dL_dweights) {
        PTRY(cudaMemcpyAsync(dL_dweights, w->dW, sizeof(double) * kMlpNW, cudaMemcpyDeviceToHost, st));
    }
    PTRY(cudaStreamSynchronize(st));
    g->C_host = g->h_S->C;
    g->t_host = g->h_S->t;
    for (int k = 0; k < 6; ++k) dL_dtheta[k] = o.lth[k];
    if (dL_dC0) *dL_dC0 = o.lC;
    for (int k = 0; k < 6; ++k)
        if (!std::isfinite(o.lth[k])) return afail(PBE_ENONFINITE, "non-finite gradient");
    return PBE_OK;
}

}  // namespace pbe

// dL/d(polynomial growth coefficients) of the last pbe_vjp (fused path, growth_form 2).
extern "C" pbe_status pbe_growth_poly_grad(pbe_grid* g, double* dL_da, int count)
{
    using namespace pbe;
    if (!g || !dL_da) return afail(PBE_EINVAL, "null argument");
    if (g->kin.growth_form != 2 || !g->adjw || !g->adjw->dpoly)
        return afail(PBE_ESTATE, "no gradient of the polynomial growth law: run pbe_vjp on the fused path first");
    const int n = g->kin.npoly * g->geo.ndim;
    if (count != n) return afail(PBE_EINVAL, "the polynomial growth law has %d coefficients (got %d)", n, count);
    cudaError_t e = cudaMemcpyAsync(dL_da, g->adjw->dpoly, sizeof(double) * n, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return afail(PBE_ECUDA, "reading the coefficient gradient failed: %s", cudaGetErrorString(e));
    return PBE_OK;
}

// The summed closure weight gradient of the last fused-path pbe_vjp of every
// grid: one launch of the weight-gradient kernel over all their rows.
extern "C" pbe_status pbe_closure_grad(pbe_grid* const* grids, int count, double* dL_dweights)
{
    using namespace pbe;
    if (!grids || count < 1 || !dL_dweights) return afail(PBE_EINVAL, "null argument or count < 1");
    pbe_grid* g0 = grids[0];
    long long R = 0;
    for (int i = 0; i < count; ++i) {
        pbe_grid* g = grids[i];
        if (!g) return afail(PBE_EINVAL, "grid %d is null", i);
        if (g->device != g0->device) return afail(PBE_EINVAL, "grid %d is on another device", i);
        if (g->kin.kind != PBE_KINETICS_MLP || !g->adjw || g->adjw->last_nrows < 0)
            return afail(PBE_ESTATE, "grid %d has no closure gradient rows: run pbe_vjp on the fused path first", i);
        if (g->mhash != g0->mhash) return afail(PBE_EINVAL, "grid %d holds other closure weights than grid 0", i);
        R += g->adjw->last_nrows;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != g0->device && cudaSetDevice(g0->device) != cudaSuccess) return afail(PBE_ECUDA, "cannot select device");
    struct Restore {
        int dev;
        ~Restore() { if (dev >= 0) cudaSetDevice(dev); }
    } restore{prev != g0->device ? prev : -1};
    AdjWork* w = g0->adjw;
    cudaStream_t st = g0->stream;
    for (int i = 0; i < count; ++i) PTRY(cudaStreamSynchronize(grids[i]->stream));
    if (w->catrows_cap < R) {
        if (grow(&w->catrows, (size_t)std::max(R, 1LL) * 6) != cudaSuccess) {
            w->catrows_cap = 0;
            cudaGetLastError();
            return afail(PBE_ENOMEM, "allocating %lld closure rows failed", R);
        }
        w->catrows_cap = R;
    }
    long long at = 0;
    for (int i = 0; i < count; ++i) {
        const long long n = grids[i]->adjw->last_nrows;
        if (n > 0)
            PTRY(cudaMemcpyAsync(w->catrows + at * 6, grids[i]->adjw->mrows, sizeof(float) * 6 * n,
                                 cudaMemcpyDeviceToDevice, st));
        at += n;
    }
    PTRY(launch_mlp_grad(w->catrows, R, g0->d_mW, g0->d_mB, w->gpart, w->dW, st));
    PTRY(cudaMemcpyAsync(dL_dweights, w->dW, sizeof(double) * kMlpNW, cudaMemcpyDeviceToHost, st));
    PTRY(cudaStreamSynchronize(st));
    return PBE_OK;
}

// Batched 1-D solves: thousands of independent instances (own grid size,
// kinetics, cooling profile and CFL-limited step count) in one persistent
// launch.  An instance is solved either by one warp or, for the costliest
// ones, by a team (all warps of a block, each a contiguous share of the
// rows).  Its distribution and stage buffer stay in shared memory for the
// whole solve, the limiter stencil's neighbours come from shared memory and
// warp shuffles, and the scalar chain runs redundantly in every lane, so an
// instance synchronizes only within its warp or block.  Blocks first pull
// team instances from one atomic queue, then their warps pull the others
// from a second one; both are ordered by estimated cost (longest first).
// The launch is captured in a CUDA graph and replayed; the schedule (warps
// per block, team instances) is chosen by pbe_batch_autotune.
//
// Moment sums are formed per segment of kSegRows rows (lane partials in row
// order, an xor butterfly over the lanes, several values sharing one) and
// the segment sums added in segment order, so results are bitwise identical
// under every schedule.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <functional>
#include <set>
#include <tuple>
#include <vector>

#include "pbe_chain.cuh"
#include "pbe_internal.h"
#include "pbe_tiles.cuh"

void pbe_set_error_message(int code, const char* msg);  // pbe_api.cu
extern "C" void pbe_batch_internal_free_vjp_work(void* w);   // pbe_batch_adjoint.cu

namespace pbe {

constexpr int kMaxBatchCells = 6144;   // largest instance accepted (shared-memory resident)

// buffer layout per instance (cell i at index i + 2, two zero ghosts below)
__host__ __device__ inline int batch_np(int N) { return 32 * ((N + 31) / 32 + 1) + 3; }

constexpr int kSegRows = 8;                                   // rows of 32 cells per moment segment
constexpr int kMaxSeg = (kMaxBatchCells / 32 + kSegRows - 1) / kSegRows;

// Butterfly sums over the warp of several values at once, bitwise equal to
// one xor butterfly (levels 16, 8, 4, 2, 1) per value: at the first levels each lane
// keeps the values of its half and sends the others, so every partial sum is
// the one the single-value butterfly forms in that lane.
//  allsum4_split: v = the sum of m[lane / 8] (lanes 0-7 m0, ..., 24-31 m3).
//  allsum2_split: v = the sum of a (lanes 0-15) or of b (lanes 16-31).
__device__ __forceinline__ double allsum4_split(const double (&m)[4])
{
    const int lane = threadIdx.x & 31;
    const bool h16 = lane & 16, h8 = lane & 8;
    const double k0 = h16 ? m[2] : m[0], k1 = h16 ? m[3] : m[1];
    const double s0 = h16 ? m[0] : m[2], s1 = h16 ? m[1] : m[3];
    const double a0 = k0 + __shfl_xor_sync(0xffffffffu, s0, 16);
    const double a1 = k1 + __shfl_xor_sync(0xffffffffu, s1, 16);
    double v = (h8 ? a1 : a0) + __shfl_xor_sync(0xffffffffu, h8 ? a0 : a1, 8);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double allsum2_split(double a, double b)
{
    const int lane = threadIdx.x & 31;
    const bool h16 = lane & 16;
    double v = (h16 ? b : a) + __shfl_xor_sync(0xffffffffu, h16 ? a : b, 16);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The moment weights are x_i^k = (2i + 1)^k (dL/2)^k: the integer powers are
// formed in integer arithmetic (exact: (2 kMaxBatchCells)^3 < 2^52) and
// converted by one addition each, the factor (dL/2)^k dL applied to the
// segment sums; the volume moment alone costs two FP64 operations a cell.
static_assert((2.0 * kMaxBatchCells) * (2.0 * kMaxBatchCells) * (2.0 * kMaxBatchCells) < 4503599627370496.0,
              "exact moment weights");

// One row of a stage (cell i = 32 r + lane): the face value of the next
// row's faces (hnext, from shared memory), the update with the flux of the
// lane to the right (shuffle), and the row's moment weights (2i + 1)^k
// (the factors (dL/2)^k dL are applied to the segment sums) added to m.  src_row: the row may
// hold cell 0, which receives the nucleation source.  A face's upwind
// difference n_{f-1} - n_{f-2} is the downwind difference of the face one
// lane to the left (lane 0: of lane 31 one row up, carried in b31), so each
// face computes one difference (the same value face_value forms).
template <int STAGE>
__device__ __forceinline__ void stage_row(const double* in, const double* old, double* out, int N, int i, double c1,
                                          double src, bool src_row, bool moms, double& hcur, double& b31,
                                          double (&m)[4])
{
    const int lane = threadIdx.x & 31;
    double v;
    if (STAGE == 0) {
        v = in[i + 2];
    } else {
        const int fn = i + 32;
        const double up = in[fn + 1], bq = in[fn + 2] - up;
        const double au = __shfl_up_sync(0xffffffffu, bq, 1);
        const double aq = lane == 0 ? b31 : au;
        b31 = __shfl_sync(0xffffffffu, bq, 31);
        const double hnext = fma(aq, psi_quot_fast(aq, bq), up);
        const double a = __shfl_down_sync(0xffffffffu, hcur, 1);
        const double b = __shfl_sync(0xffffffffu, hnext, 0);
        const double hright = lane == 31 ? b : a;
        v = fma(c1, hcur - hright, in[i + 2]);
        if (src_row && i == 0) v += src;
        if (STAGE == 2) v = fma(0.5, old[i + 2], 0.5 * v);
        if (i < N) out[i + 2] = v;
        hcur = hnext;
    }
    if (i < N) {
        const long long w1 = 2LL * i + 1, w3 = w1 * w1 * w1;
        if (moms) {
            m[0] += v;
            m[1] = fma(exact_int_double(w1), v, m[1]);
            m[2] = fma(exact_int_double(w1 * w1), v, m[2]);
        }
        m[3] = fma(exact_int_double(w3), v, m[3]);
    }
}

// The lane partials of one segment of a stage (rows r0 .. r0 + nr - 1).
template <int STAGE>
__device__ __forceinline__ void stage_segment(const double* in, const double* old, double* out, int N, int r0, int nr,
                                              double c1, double src, double d1, bool moms, double& hcur,
                                              double& b31, double (&m)[4])
{
    const int lane = threadIdx.x & 31;
    m[0] = 0.0; m[1] = 0.0; m[2] = 0.0; m[3] = 0.0;
    const int i0 = 32 * r0 + lane;
    if (nr == kSegRows) {
#pragma unroll
        for (int j = 0; j < kSegRows; ++j)
            stage_row<STAGE>(in, old, out, N, i0 + 32 * j, c1, src, j == 0 && r0 == 0, moms, hcur, b31, m);
    } else {
        for (int j = 0; j < nr; ++j)
            stage_row<STAGE>(in, old, out, N, i0 + 32 * j, c1, src, j == 0 && r0 == 0, moms, hcur, b31, m);
    }
}

// One stage over the segments [p0, p1) of an instance of R rows (32 cells a
// row, one a lane): STAGE 1 writes n1 = n + dt L(n), STAGE 2 writes
// n = n/2 + (n1 + dt L(n1))/2, STAGE 0 only measures `in`.  The face values
// come from shared memory and the lane to the right (shuffle).  Segment sums
// of the moment weights (all four with `moms`, else mu3 alone) go to
// seg[4p + k] (when seg is non-null) or are added to tot in segment order.
template <int STAGE>
__device__ __forceinline__ void warp_stage(const double* in, const double* old, double* out, int N, int R, int p0,
                                           int p1, double c1, double src, double d1, bool moms, double* seg,
                                           double (&tot)[4])
{
    const int lane = threadIdx.x & 31;
    if (p0 >= p1) return;
    // face f lies between cells f-1 (upwind) and f: (n_{f-2}, n_{f-1}, n_f) = in[f], in[f+1], in[f+2]
    const int f0 = 32 * p0 * kSegRows + lane;
    double hcur = 0.0, b31 = 0.0;
    if (STAGE != 0) {
        hcur = face_value<true>(in[f0], in[f0 + 1], in[f0 + 2]);
        b31 = __shfl_sync(0xffffffffu, in[f0 + 2] - in[f0 + 1], 31);
    }
    double m[4];
    // the weights' factors (dL/2)^k dL
    const double hd = 0.5 * d1, f1 = d1 * hd, f2 = f1 * hd, f3 = f2 * hd;
    if (moms) {
        // lane group k = lane / 8 carries moment k
        const int k8 = lane >> 3;
        const double fk = k8 == 0 ? d1 : (k8 == 1 ? f1 : (k8 == 2 ? f2 : f3));
        double acc = 0.0;
        for (int p = p0; p < p1; ++p) {
            const int r0 = p * kSegRows;
            stage_segment<STAGE>(in, old, out, N, r0, min(kSegRows, R - r0), c1, src, d1, true, hcur, b31, m);
            const double v = allsum4_split(m) * fk;
            if (seg) {
                if ((lane & 7) == 0) seg[4 * p + (lane >> 3)] = v;
            } else {
                acc += v;
            }
        }
        if (!seg) {
#pragma unroll
            for (int k = 0; k < 4; ++k) tot[k] += __shfl_sync(0xffffffffu, acc, 8 * k);
        }
        return;
    }
    // mu3 alone: segments in pairs
    double acc = 0.0;
    for (int p = p0; p < p1; p += 2) {
        const int r0 = p * kSegRows;
        stage_segment<STAGE>(in, old, out, N, r0, min(kSegRows, R - r0), c1, src, d1, false, hcur, b31, m);
        const double a = m[3];
        double b = 0.0;
        if (p + 1 < p1) {
            stage_segment<STAGE>(in, old, out, N, r0 + kSegRows, min(kSegRows, R - r0 - kSegRows), c1, src, d1,
                                 false, hcur, b31, m);
            b = m[3];
        }
        const double v = allsum2_split(a, b);
        const double sa = __shfl_sync(0xffffffffu, v, 0) * f3, sb = __shfl_sync(0xffffffffu, v, 16) * f3;
        if (seg) {
            if (lane == 0) seg[4 * p + 3] = sa;
            if (lane == 16 && p + 1 < p1) seg[4 * (p + 1) + 3] = sb;
        } else {
            acc += sa;
            if (p + 1 < p1) acc += sb;
        }
    }
    if (!seg) tot[3] += acc;
}

// Block-shared scratch of a team: segment sums, two buffers used alternately
// so that one block barrier per stage suffices.
struct TeamSm {
    double seg[2][kMaxSeg * 4];
};

// A stage of one instance by one warp (TEAM false: all segments) or by the
// block (TEAM true: this warp's segments, then the segment sums of all warps
// added in order after a block barrier, which also orders this stage's
// writes before the next stage's reads).  Returns the sums in m.
template <int STAGE, bool TEAM, int WPB>
__device__ __forceinline__ void inst_stage(const double* in, const double* old, double* out, int N, int R, double c1,
                                           double src, double d1, bool moms, TeamSm* ts, int& par, double (&m)[4])
{
    for (int k = 0; k < 4; ++k) m[k] = 0.0;
    const int P = (R + kSegRows - 1) / kSegRows;
    if (!TEAM) {
        warp_stage<STAGE>(in, old, out, N, R, 0, P, c1, src, d1, moms, nullptr, m);
        __syncwarp();
        return;
    }
    const int warp = threadIdx.x >> 5;
    double* seg = ts->seg[par];
    warp_stage<STAGE>(in, old, out, N, R, (warp * P) / WPB, ((warp + 1) * P) / WPB, c1, src, d1, moms, seg, m);
    __syncthreads();
    for (int p = 0; p < P; ++p) {
        if (moms) { m[0] += seg[4 * p]; m[1] += seg[4 * p + 1]; m[2] += seg[4 * p + 2]; }
        m[3] += seg[4 * p + 3];
    }
    par ^= 1;
}

// The rates of one instance at (C, t): the power law (or fixed rates), or,
// in batches with the learned closure (MLP), the closure with its moment-
// ratio input V / mu0 and its fallback to the power law.
template <bool MLP>
__device__ __forceinline__ void batch_rates(const Kin& K, double C, double t, double ratio, double& G1, double& B)
{
    double G2;
    if constexpr (MLP) kinetics_warp_r(K, C, t, ratio, G1, G2, B);
    else kinetics_warp<false>(K, C, t, G1, G2, B);
}

// One instance, solved by one warp (TEAM false) or by all WPB warps of the
// block (TEAM true).  nb, n1b: the instance's state and stage buffers in
// shared memory (cell i at index i + 2, two zero ghosts below).
template <bool TEAM, int WPB, bool MLP>
__device__ __forceinline__ void run_instance(int id, const BatchInst* __restrict__ inst, double* state, double* Cst,
                                             double* tst, const double* t_out, int n_out, double* rows,
                                             long long* steps_out, int* status_out, long long max_steps, double* nb,
                                             double* n1b, TeamSm* ts)
{
    const int lane = threadIdx.x & 31;
    const int tid = TEAM ? (int)threadIdx.x : lane, nthr = TEAM ? WPB * 32 : 32;
    const bool writer = TEAM ? threadIdx.x == 0 : lane == 0;
    int par = 0;
    const Kin K = inst[id].K;
    const Geom g = inst[id].g;
    const long long off = inst[id].offset;
    const int N = g.N1, R = inst[id].rows;
    const int np = batch_np(N);
    for (int k = tid; k < np; k += nthr) {
        const int i = k - 2;
        nb[k] = (i >= 0 && i < N) ? state[off + i] : 0.0;
        n1b[k] = 0.0;
    }
    if (TEAM) __syncthreads();
    else __syncwarp();
    // scalar state (identical in every lane of the warp or team)
    Scal s;
    s.C = Cst[id];
    s.t = tst[id];
    s.steps = 0; s.status = 0; s.done = 0; s.out_idx = 0; s.n_out = n_out; s.max_steps = max_steps;
    double m[4];
    inst_stage<0, TEAM, WPB>(nb, nb, nb, N, R, 0.0, 0.0, g.d1, true, ts, par, m);
    s.V0 = m[3];
    double M0 = m[0];   // mu0 of the current state (the closure's input ratio V / mu0)
    double* my_rows = rows + (size_t)id * n_out * 6;
    // power law: the stage-1 chain's evaluation, for the series of the next
    // step's rates (both at the step's end time t_new), and that time's
    // temperature and solubility
    RateCarry rc;
    KinT tc{0.0, 0.0};
    if (!MLP) rate_carry_init(rc, K);
    if (!isfinite(m[0]) || !isfinite(m[3]) || !isfinite(s.C)) {
        s.status = PBE_ENONFINITE;
        s.done = 1;
    } else {
        while (s.out_idx < n_out && t_out[s.out_idx] == s.t) {
            if (writer) {
                double* row = my_rows + (size_t)s.out_idx * 6;
                row[0] = s.t; row[1] = m[0]; row[2] = m[1]; row[3] = m[2]; row[4] = m[3]; row[5] = s.C;
            }
            s.out_idx += 1;
        }
        if (s.out_idx >= n_out) s.done = 1;
    }
    if (!s.done) {
        double G1, B, dt, t_new;
        batch_rates<MLP>(K, s.C, s.t, MLP ? s.V0 / M0 : 0.0, G1, B);
        s.clipped = timestep_fast(K, g, G1, 0.0, s.t, t_out[s.out_idx], dt, t_new);
        s.G1a = G1; s.Ba = B; s.dt = dt; s.t_new = t_new;
        if (!isfinite(G1) || !isfinite(B) || !isfinite(dt)) { s.status = PBE_ENONFINITE; s.done = 1; }
    }
    while (!s.done) {
        // stage 1: n1 = n + dt L(n)
        inst_stage<1, TEAM, WPB>(nb, nb, n1b, N, R, s.G1a * s.dt * g.inv_d1, s.dt * s.Ba * g.inv_d1, g.d1, MLP, ts,
                                 par, m);
        const double V1 = m[3];
        const double C1 = fma(-K.kappa, V1 - s.V0, s.C);
        {
            double G1, B;
            if (MLP) {
                batch_rates<MLP>(K, C1, s.t_new, V1 / m[0], G1, B);
            } else {   // power law: the step's end time once, the evaluation kept for the series
                tc = kin_temperature(K, s.t_new);
                double G2, L, rec[2];
                kinetics_warp_T<false>(K, C1, tc, G1, G2, B, &L, nullptr, rec);
                rate_carry_keep(rc, K, G1, G2, B, L, rec);
            }
            s.G1b = G1; s.Bb = B;
            if (!isfinite(V1) || !isfinite(G1) || !isfinite(B)) { s.status = PBE_ENONFINITE; s.done = 1; break; }
        }
        // stage 2: n = n/2 + (n1 + dt L(n1))/2
        const bool moms = s.clipped;
        inst_stage<2, TEAM, WPB>(n1b, nb, nb, N, R, s.G1b * s.dt * g.inv_d1, s.dt * s.Bb * g.inv_d1, g.d1,
                                 moms || MLP, ts, par, m);
        const double V2 = m[3];
        if (MLP) M0 = m[0];
        s.C = fma(-K.kappa, V2 - s.V0, s.C);
        s.t = s.t_new;
        s.V0 = V2;
        s.steps += 1;
        if (!isfinite(V2) || !isfinite(s.C)) { s.status = PBE_ENONFINITE; s.done = 1; break; }
        if (moms) {
            if (writer) {
                double* row = my_rows + (size_t)s.out_idx * 6;
                row[0] = s.t; row[1] = m[0]; row[2] = m[1]; row[3] = m[2]; row[4] = m[3]; row[5] = s.C;
            }
            s.out_idx += 1;
        }
        if (s.out_idx >= n_out) { s.done = 1; break; }
        if (s.steps >= max_steps) { s.status = PBE_ETIMEOUT; s.done = 1; break; }
        double G1, B, dt, t_new;
        if (MLP) {
            batch_rates<MLP>(K, s.C, s.t, s.V0 / M0, G1, B);
        } else {   // the same time as the stage-1 evaluation: the series where it applies
            double G2, L;
            if (!rates_by_series(rc, s.C, tc.cs, 1, G1, G2, B, L)) kinetics_warp_T<false>(K, s.C, tc, G1, G2, B);
        }
        s.clipped = timestep_fast(K, g, G1, 0.0, s.t, t_out[s.out_idx], dt, t_new);
        s.G1a = G1; s.Ba = B; s.dt = dt; s.t_new = t_new;
        if (!isfinite(G1) || !isfinite(B) || !isfinite(dt)) { s.status = PBE_ENONFINITE; s.done = 1; }
    }
    if (TEAM) __syncthreads();
    else __syncwarp();
    for (int i = tid; i < N; i += nthr) state[off + i] = nb[i + 2];
    if (writer) {
        Cst[id] = s.C;
        tst[id] = s.t;
        steps_out[id] = s.steps;
        status_out[id] = s.status;
    }
    if (TEAM) __syncthreads();
    else __syncwarp();
}

// The batch kernel.  order[0..nteam) are the team instances (each solved by
// a whole block, pulled from queue[0]); order[nteam..count) the others (one
// per warp, from queue[1]).  np_slot: doubles per buffer of a warp's slice
// (two buffers a warp); a team uses the block's whole allocation, nb at the
// start and n1b half way.
template <int WPB, bool MLP>
__global__ void __maxnreg__(168) k_batch1d(const BatchInst* __restrict__ inst, const int* __restrict__ order,
                                                      int count, int nteam, double* state, double* Cst, double* tst,
                                                      const double* t_out, int n_out, double* rows,
                                                      long long* steps_out, int* status_out, unsigned int* queue,
                                                      int np_slot, long long max_steps)
{
    extern __shared__ double smem[];
    __shared__ TeamSm ts;
    __shared__ int s_idx;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (nteam > 0) {
        for (;;) {
            if (threadIdx.x == 0) s_idx = (int)atomicAdd(queue, 1u);
            __syncthreads();
            const int idx = s_idx;
            __syncthreads();
            if (idx >= nteam) break;
            run_instance<true, WPB, MLP>(order[idx], inst, state, Cst, tst, t_out, n_out, rows, steps_out, status_out,
                                    max_steps, smem, smem + (size_t)WPB * np_slot, &ts);
        }
    }
    double* nb = smem + (size_t)warp * 2 * np_slot;
    double* n1b = nb + np_slot;
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = nteam + (int)atomicAdd(queue + 1, 1u);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= count) break;
        run_instance<false, WPB, MLP>(order[idx], inst, state, Cst, tst, t_out, n_out, rows, steps_out, status_out,
                                 max_steps, nb, n1b, &ts);
    }
}

}  // namespace pbe

using namespace pbe;

struct pbe_batch {
    int device;
    int count;
    cudaStream_t stream;
    std::vector<long long> offsets;   // count + 1
    std::vector<double> C0, t0;
    long long total_cells;
    int np_max;
    int wpb;                          // warps per block
    int nteam;                        // the nteam costliest instances are team instances ...
    int wcells;                       // ... and so is every instance of more than wcells cells
    int nteam_default;                // the cost heuristic's team count (autotune's starting point)
    int nmax;                         // cells of the largest instance
    std::vector<double> cost;         // estimated cost of each instance (cells x CFL steps)
    std::vector<int> ncells;
    std::vector<int> by_cost;         // instance ids by estimated cost, longest first
    std::vector<int> sizes_desc;      // the distinct instance sizes, largest first
    std::vector<int> order_h;         // the queue order uploaded to d_order ...
    int order_nteam, order_wcells;    // ... for this team selection (-1: none yet)
    int vjp_warps;                    // warps per instance of pbe_batch_vjp (0: chosen from the batch size)
    int vjp_blocks;                   // resident teams per SM of pbe_batch_vjp (0: as many as fit)
    int power_law;                    // every instance has power-law kinetics and the polynomial solubility
    int mlp;                          // some instance has the learned closure (the MLP kernel variant)
    int closure_set;                  // its weights are on the device (pbe_batch_set_closure)
    std::vector<BatchInst> h_inst;    // host copy of the instance descriptors
    __nv_bfloat16* d_mW;              // the batch's closure weights (bf16 matrices, fp32 biases)
    float* d_mB;
    void* vjp_work;                   // pbe_batch_vjp's device scratch (pbe_batch_adjoint.cu)
    long long max_steps;
    BatchInst* d_inst;
    int* d_order;
    double* d_state;
    double *d_C, *d_t;
    long long* d_steps;
    int* d_status;
    unsigned int* d_queue;
    double* d_tout;
    double* d_rows;
    int tout_cap;
    cudaGraphExec_t exec;
    int exec_wpb, exec_nteam, exec_wcells, exec_nout;
    long long* h_steps;
    int* h_status;
};

namespace {

pbe_status bfail(pbe_status code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    pbe_set_error_message(code, buf);
    return code;
}

#define BTRY(call)                                                                                     \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return bfail(PBE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

const void* batch_kernel(int wpb, bool mlp = false)
{
    switch (wpb) {
        case 1: return mlp ? (const void*)k_batch1d<1, true> : (const void*)k_batch1d<1, false>;
        case 2: return mlp ? (const void*)k_batch1d<2, true> : (const void*)k_batch1d<2, false>;
        case 3: return mlp ? (const void*)k_batch1d<3, true> : (const void*)k_batch1d<3, false>;
        case 4: return mlp ? (const void*)k_batch1d<4, true> : (const void*)k_batch1d<4, false>;
        case 6: return mlp ? (const void*)k_batch1d<6, true> : (const void*)k_batch1d<6, false>;
        case 8: return mlp ? (const void*)k_batch1d<8, true> : (const void*)k_batch1d<8, false>;
        default: return nullptr;
    }
}

// The team instances of a selection (the nteam costliest, and every one of
// more than wcells cells): how many, and the largest team and warp instance.
struct TeamSplit {
    int teams, team_nmax, warp_nmax;
};

TeamSplit team_split(const pbe_batch* b, int nteam, int wcells)
{
    TeamSplit t{0, 0, 0};
    for (int j = 0; j < b->count; ++j) {
        const int N = b->ncells[b->by_cost[j]];
        if (j < nteam || N > wcells) {
            ++t.teams;
            t.team_nmax = std::max(t.team_nmax, N);
        } else {
            t.warp_nmax = std::max(t.warp_nmax, N);
        }
    }
    return t;
}

// Doubles per buffer of a warp's shared-memory slice under a schedule: large
// enough for every warp instance, and (the block's 2 * wpb buffers split in
// two halves) for every team instance.
int batch_np_slot(const pbe_batch* b, int wpb, int nteam, int wcells)
{
    const TeamSplit t = team_split(b, nteam, wcells);
    int np = t.warp_nmax > 0 ? batch_np(t.warp_nmax) : 0;
    if (t.teams > 0) np = std::max(np, (batch_np(t.team_nmax) + wpb - 1) / wpb);
    return np;
}

size_t batch_smem(const pbe_batch* b, int wpb, int nteam, int wcells)
{
    return (size_t)wpb * 2 * batch_np_slot(b, wpb, nteam, wcells) * sizeof(double);
}

// The queue order of a team selection: the team instances, then the others,
// each part by estimated cost, longest first.
cudaError_t upload_order(pbe_batch* b, int nteam, int wcells)
{
    if (b->order_nteam == nteam && b->order_wcells == wcells) return cudaSuccess;
    std::vector<int>& o = b->order_h;
    o.clear();
    for (int j = 0; j < b->count; ++j)
        if (j < nteam || b->ncells[b->by_cost[j]] > wcells) o.push_back(b->by_cost[j]);
    for (int j = 0; j < b->count; ++j)
        if (!(j < nteam || b->ncells[b->by_cost[j]] > wcells)) o.push_back(b->by_cost[j]);
    cudaError_t e = cudaStreamSynchronize(b->stream);   // no launch in flight reads the old order
    if (e == cudaSuccess) e = cudaMemcpy(b->d_order, o.data(), sizeof(int) * b->count, cudaMemcpyHostToDevice);
    b->order_nteam = e == cudaSuccess ? nteam : -1;
    b->order_wcells = wcells;
    return e;
}

// Launch of one batch solve under a schedule (the order must be uploaded).
cudaError_t launch_batch(pbe_batch* b, int wpb, int nteam, int wcells, int n_out, cudaStream_t st)
{
    const void* fn = batch_kernel(wpb, b->mlp != 0);
    size_t smem = batch_smem(b, wpb, nteam, wcells);
    int np_slot = batch_np_slot(b, wpb, nteam, wcells);
    int teams = team_split(b, nteam, wcells).teams;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, wpb * 32, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) return e;
    int blocks = occ * sms;
    const int need = teams + (b->count - teams + wpb - 1) / wpb;
    if (blocks > need) blocks = need;
    e = cudaMemsetAsync(b->d_queue, 0, 2 * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    void* args[] = {&b->d_inst, &b->d_order, &b->count, &teams, &b->d_state, &b->d_C, &b->d_t, &b->d_tout, &n_out,
                    &b->d_rows, &b->d_steps, &b->d_status, &b->d_queue, &np_slot, &b->max_steps};
    return cudaLaunchKernel(fn, blocks, wpb * 32, args, smem, st);
}

int max_block_smem(const pbe_batch* b)
{
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
    return maxsm - (int)sizeof(TeamSm) - 64;
}

bool schedule_fits(const pbe_batch* b, int wpb, int nteam, int wcells)
{
    return batch_smem(b, wpb, nteam, wcells) <= (size_t)max_block_smem(b);
}

// Blocks per SM that a schedule's shared memory (and the registers) allow.
int blocks_per_sm(const pbe_batch* b, int wpb, int nteam, int wcells)
{
    const void* fn = batch_kernel(wpb, b->mlp != 0);
    int occ = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_block_smem(b)) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, wpb * 32, batch_smem(b, wpb, nteam, wcells)) !=
            cudaSuccess)
        occ = 0;
    return occ;
}

// The largest size cut at or below wcells (a distinct instance size, or 0)
// with which the schedule fits; -1 when none does.
int fitting_wcells(const pbe_batch* b, int wpb, int nteam, int wcells)
{
    for (int N : b->sizes_desc)
        if (N <= wcells && schedule_fits(b, wpb, nteam, N)) return N;
    return schedule_fits(b, wpb, nteam, 0) ? 0 : -1;
}

pbe_status ensure_tout(pbe_batch* b, int n_out)
{
    if (n_out <= b->tout_cap) return PBE_OK;
    BTRY(cudaStreamSynchronize(b->stream));
    cudaFree(b->d_tout);
    cudaFree(b->d_rows);
    b->d_tout = nullptr;
    b->d_rows = nullptr;
    b->tout_cap = 0;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (cudaMalloc(&b->d_tout, sizeof(double) * n_out) != cudaSuccess ||
        cudaMalloc(&b->d_rows, sizeof(double) * 6 * (size_t)n_out * b->count) != cudaSuccess)
        return bfail(PBE_ENOMEM, "allocating %d output rows for %d instances failed", n_out, b->count);
    b->tout_cap = n_out;
    return PBE_OK;
}

pbe_status check_times(const pbe_batch* b, const double* t_out, int n_out)
{
    if (!t_out || n_out < 1) return bfail(PBE_EINVAL, "need at least one output time");
    for (int j = 0; j < n_out; ++j)
        if (!std::isfinite(t_out[j]) || (j > 0 && !(t_out[j] > t_out[j - 1])))
            return bfail(PBE_EINVAL, "t_out must be strictly increasing and finite (index %d)", j);
    (void)b;
    return PBE_OK;
}

// Graph of one batch solve (queue reset + persistent kernel), rebuilt when the
// configuration or the number of output times changes.
pbe_status run_batch(pbe_batch* b, int n_out)
{
    if (!b->exec || b->exec_wpb != b->wpb || b->exec_nteam != b->nteam || b->exec_wcells != b->wcells ||
        b->exec_nout != n_out) {
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        cudaStream_t cap;
        BTRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
        cudaError_t le = cudaSuccess;
        if (e == cudaSuccess) {
            le = launch_batch(b, b->wpb, b->nteam, b->wcells, n_out, cap);
            e = cudaStreamEndCapture(cap, &graph);
        }
        if (e == cudaSuccess) e = le;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return bfail(PBE_ECUDA, "building the batch graph failed: %s", cudaGetErrorString(e));
        }
        b->exec_wpb = b->wpb;
        b->exec_nteam = b->nteam;
        b->exec_wcells = b->wcells;
        b->exec_nout = n_out;
    }
    BTRY(cudaGraphLaunch(b->exec, b->stream));
    return PBE_OK;
}

pbe_status collect_status(pbe_batch* b, int64_t* total_steps)
{
    BTRY(cudaMemcpyAsync(b->h_steps, b->d_steps, sizeof(long long) * b->count, cudaMemcpyDeviceToHost, b->stream));
    BTRY(cudaMemcpyAsync(b->h_status, b->d_status, sizeof(int) * b->count, cudaMemcpyDeviceToHost, b->stream));
    BTRY(cudaStreamSynchronize(b->stream));
    long long tot = 0;
    for (int i = 0; i < b->count; ++i) tot += b->h_steps[i];
    if (total_steps) *total_steps = tot;
    for (int i = 0; i < b->count; ++i) {
        if (b->h_status[i] == PBE_ENONFINITE) return bfail(PBE_ENONFINITE, "instance %d: non-finite value", i);
        if (b->h_status[i] == PBE_ETIMEOUT) return bfail(PBE_ETIMEOUT, "instance %d: step budget exhausted", i);
        if (b->h_status[i] != PBE_OK) return bfail(b->h_status[i], "instance %d: device status %d", i, b->h_status[i]);
    }
    return PBE_OK;
}

}  // namespace

extern "C" {

pbe_status pbe_batch_create(pbe_batch** out, const pbe_instance* inst, int count)
{
    if (!out || !inst) return bfail(PBE_EINVAL, "null argument");
    *out = nullptr;
    if (count < 1) return bfail(PBE_EINVAL, "count must be >= 1");
    std::vector<BatchInst> h(count);
    std::vector<double> cost(count);
    pbe_batch* b = new pbe_batch();
    b->count = count;
    b->offsets.resize(count + 1);
    b->C0.resize(count);
    b->t0.resize(count);
    b->offsets[0] = 0;
    int nmax = 1;
    bool power_law = true;
    for (int i = 0; i < count; ++i) {
        const pbe_instance& p = inst[i];
        const pbe_kinetics* k = &p.kin;
        if (p.ncells < 1 || p.ncells > kMaxBatchCells) {
            delete b;
            return bfail(PBE_EINVAL, "instance %d: ncells = %lld outside [1, %d]", i, (long long)p.ncells, kMaxBatchCells);
        }
        if (!(p.lmax > 0.0) || !std::isfinite(p.lmax) || !std::isfinite(p.C0) || !std::isfinite(p.t0) ||
            !(k->cfl > 0.0 && k->cfl <= 1.0) || !(k->t_cool > 0.0) ||
            (k->kind != PBE_KINETICS_POWER_LAW && k->kind != PBE_KINETICS_FIXED && k->kind != PBE_KINETICS_MLP) ||
            k->kg[0] < 0 || k->kb < 0 || k->scheme != PBE_SCHEME_SSPRK2 ||
            (k->growth_form != 0 && k->growth_form != 1) || (k->solubility_form != 0 && k->solubility_form != 1) ||
            (k->kind == PBE_KINETICS_MLP && k->growth_form != 0)) {
            // (the learned closure falls back to the power law: growth_form 0)
            delete b;
            return bfail(PBE_EINVAL, "instance %d: invalid parameters", i);
        }
        if (check_kinetic_values(k) != PBE_OK) {
            delete b;
            return bfail(PBE_EINVAL, "instance %d: %s", i, pbe_last_error());
        }
        BatchInst& d = h[i];
        memset(&d, 0, sizeof(d));
        d.K.kind = k->kind; d.K.ndim = 1;
        d.K.kg1 = k->kg[0]; d.K.g1 = k->g[0]; d.K.kg2 = 0.0; d.K.g2 = 1.0; d.K.kb = k->kb; d.K.b = k->b;
        d.K.cs0 = k->csat[0]; d.K.cs1 = k->csat[1]; d.K.cs2 = k->csat[2];
        d.K.T0 = k->T0; d.K.T1 = k->T1; d.K.t_cool = k->t_cool; d.K.kappa = k->kappa; d.K.cfl = k->cfl;
        d.K.lkg1 = std::log(k->kg[0]); d.K.lkg2 = -INFINITY; d.K.lkb = std::log(k->kb);
        d.K.inv_tcool = 1.0 / k->t_cool;
        d.K.growth_form = k->growth_form;
        power_law = power_law && k->growth_form == 0 && k->solubility_form == 0 && k->kind != PBE_KINETICS_MLP;
        if (k->kind == PBE_KINETICS_MLP) b->mlp = 1;
        d.K.solubility_form = k->solubility_form;
        d.K.ea1 = k->ea[0];
        d.g.ndim = 1; d.g.N1 = (int)p.ncells; d.g.N2 = 1; d.g.d1 = p.lmax / (double)p.ncells; d.g.d2 = 1.0;
        d.g.inv_d1 = 1.0 / d.g.d1; d.g.inv_d2 = 1.0;
        d.offset = b->offsets[i];
        d.rows = (int)((p.ncells + 31) / 32);
        b->offsets[i + 1] = b->offsets[i] + p.ncells;
        b->C0[i] = p.C0;
        b->t0[i] = p.t0;
        nmax = std::max(nmax, (int)p.ncells);
        // scheduling estimate (longest first): cells x CFL steps at the peak
        // supersaturation the cooling alone would give
        double cs0 = k->csat[0] + k->csat[1] * k->T0 + k->csat[2] * k->T0 * k->T0;
        double cs1 = k->csat[0] + k->csat[1] * k->T1 + k->csat[2] * k->T1 * k->T1;
        double smax = std::max(std::max(p.C0 / cs0, p.C0 / cs1) - 1.0, 0.0);
        double G = k->kind == PBE_KINETICS_FIXED ? k->kg[0] : k->kg[0] * std::pow(smax, k->g[0]);
        cost[i] = (double)p.ncells * (1.0 + G * k->t_cool / (k->cfl * d.g.d1));
    }
    b->total_cells = b->offsets[count];
    b->power_law = power_law ? 1 : 0;
    b->np_max = batch_np(nmax);
    b->max_steps = 1000000;
    b->cost = cost;
    b->nmax = nmax;
    b->h_inst = h;
    b->ncells.resize(count);
    for (int i = 0; i < count; ++i) b->ncells[i] = h[i].g.N1;
    b->by_cost.resize(count);
    std::iota(b->by_cost.begin(), b->by_cost.end(), 0);
    std::stable_sort(b->by_cost.begin(), b->by_cost.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    b->sizes_desc = b->ncells;
    std::sort(b->sizes_desc.begin(), b->sizes_desc.end(), std::greater<int>());
    b->sizes_desc.erase(std::unique(b->sizes_desc.begin(), b->sizes_desc.end()), b->sizes_desc.end());
    b->order_nteam = -1;
    b->order_wcells = -1;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return bfail(PBE_ECUDA, "no CUDA device available");
    }
    // default schedule: 3 warps a block; team instances: every instance whose
    // estimated cost is above the mean load of a warp (the warps the launch
    // keeps resident), i.e. that one warp alone would make the launch's tail
    {
        int sms = 1;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
        const int wpb = 3;
        const int warps = std::max(blocks_per_sm(b, wpb, 0, kMaxBatchCells), 1) * wpb * std::max(sms, 1);
        double total = 0.0;
        for (int i = 0; i < count; ++i) total += cost[i];
        int nt = 0;
        for (int i = 0; i < count; ++i) nt += cost[i] > total / warps;
        b->wpb = wpb;
        b->nteam = nt;
        b->nteam_default = nt;
        b->wcells = fitting_wcells(b, wpb, nt, kMaxBatchCells);   // fits at wcells = 0 at the latest
    }
    bool ok = cudaMalloc(&b->d_inst, sizeof(BatchInst) * count) == cudaSuccess &&
              cudaMalloc(&b->d_order, sizeof(int) * count) == cudaSuccess &&
              cudaMalloc(&b->d_state, sizeof(double) * b->total_cells) == cudaSuccess &&
              cudaMalloc(&b->d_C, sizeof(double) * count) == cudaSuccess &&
              cudaMalloc(&b->d_t, sizeof(double) * count) == cudaSuccess &&
              cudaMalloc(&b->d_steps, sizeof(long long) * count) == cudaSuccess &&
              cudaMalloc(&b->d_status, sizeof(int) * count) == cudaSuccess &&
              cudaMalloc(&b->d_queue, 2 * sizeof(unsigned int)) == cudaSuccess &&
              cudaMallocHost(&b->h_steps, sizeof(long long) * count) == cudaSuccess &&
              cudaMallocHost(&b->h_status, sizeof(int) * count) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        pbe_batch_destroy(b);
        return bfail(PBE_ENOMEM, "allocating the batch failed");
    }
    if (cudaMemcpy(b->d_inst, h.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        upload_order(b, b->nteam, b->wcells) != cudaSuccess ||
        cudaMemset(b->d_state, 0, sizeof(double) * b->total_cells) != cudaSuccess ||
        cudaMemcpy(b->d_C, b->C0.data(), sizeof(double) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_t, b->t0.data(), sizeof(double) * count, cudaMemcpyHostToDevice) != cudaSuccess) {
        pbe_batch_destroy(b);
        return bfail(PBE_ECUDA, "initialising the batch failed");
    }
    *out = b;
    return PBE_OK;
}

pbe_status pbe_batch_destroy(pbe_batch* b)
{
    if (!b) return PBE_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    pbe_batch_internal_free_vjp_work(b->vjp_work);
    cudaFree(b->d_mW); cudaFree(b->d_mB);
    cudaFree(b->d_inst); cudaFree(b->d_order); cudaFree(b->d_state); cudaFree(b->d_C); cudaFree(b->d_t);
    cudaFree(b->d_steps); cudaFree(b->d_status); cudaFree(b->d_queue); cudaFree(b->d_tout); cudaFree(b->d_rows);
    cudaFreeHost(b->h_steps); cudaFreeHost(b->h_status);
    delete b;
    return PBE_OK;
}

pbe_status pbe_batch_set_stream(pbe_batch* b, void* stream)
{
    if (!b) return bfail(PBE_EINVAL, "null batch");
    b->stream = (cudaStream_t)stream;
    return PBE_OK;
}

pbe_status pbe_batch_offsets(pbe_batch* b, int64_t* offsets)
{
    if (!b || !offsets) return bfail(PBE_EINVAL, "null argument");
    for (int i = 0; i <= b->count; ++i) offsets[i] = b->offsets[i];
    return PBE_OK;
}

pbe_status pbe_batch_set_state(pbe_batch* b, const double* n_packed, int mem)
{
    if (!b || !n_packed) return bfail(PBE_EINVAL, "null argument");
    cudaMemcpyKind kd = mem == PBE_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    BTRY(cudaMemcpyAsync(b->d_state, n_packed, sizeof(double) * b->total_cells, kd, b->stream));
    BTRY(cudaMemcpyAsync(b->d_C, b->C0.data(), sizeof(double) * b->count, cudaMemcpyHostToDevice, b->stream));
    BTRY(cudaMemcpyAsync(b->d_t, b->t0.data(), sizeof(double) * b->count, cudaMemcpyHostToDevice, b->stream));
    BTRY(cudaStreamSynchronize(b->stream));  // C0/t0 are pageable host vectors
    return PBE_OK;
}

pbe_status pbe_batch_get_state(pbe_batch* b, double* n_packed, double* C, double* t, int mem)
{
    if (!b) return bfail(PBE_EINVAL, "null batch");
    cudaMemcpyKind kd = mem == PBE_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (n_packed) BTRY(cudaMemcpyAsync(n_packed, b->d_state, sizeof(double) * b->total_cells, kd, b->stream));
    if (C) BTRY(cudaMemcpyAsync(C, b->d_C, sizeof(double) * b->count, kd, b->stream));
    if (t) BTRY(cudaMemcpyAsync(t, b->d_t, sizeof(double) * b->count, kd, b->stream));
    BTRY(cudaStreamSynchronize(b->stream));
    return PBE_OK;
}

// accessor for the batched adjoint (pbe_batch_adjoint.cu); not part of the public header
pbe_status pbe_batch_internal_view(pbe_batch* b, const void** inst, const int** order, int* count, double** state,
                                   double** C, double** t, int* np_max, int* device, void** stream)
{
    *inst = b->d_inst;
    *order = b->d_order;
    *count = b->count;
    *state = b->d_state;
    *C = b->d_C;
    *t = b->d_t;
    *np_max = b->np_max;
    *device = b->device;
    *stream = (void*)b->stream;
    return PBE_OK;
}

// accessors for the batched adjoint; not part of the public header
int pbe_batch_internal_vjp_warps(const pbe_batch* b) { return b->vjp_warps; }
int pbe_batch_internal_vjp_blocks(const pbe_batch* b) { return b->vjp_blocks; }
int pbe_batch_internal_power_law(const pbe_batch* b) { return b->power_law; }
void** pbe_batch_internal_vjp_work(pbe_batch* b) { return &b->vjp_work; }

pbe_status pbe_batch_set_vjp_schedule(pbe_batch* b, int warps, int blocks_per_sm)
{
    if (!b) return bfail(PBE_EINVAL, "null batch");
    if (warps != 0 && warps != 1 && warps != 2 && warps != 4 && warps != 8)
        return bfail(PBE_EINVAL, "warps per instance must be 0 (automatic), 1, 2, 4 or 8");
    if (blocks_per_sm < 0 || blocks_per_sm > 32)
        return bfail(PBE_EINVAL, "blocks_per_sm must be 0 (as many as fit) .. 32");
    b->vjp_warps = warps;
    b->vjp_blocks = blocks_per_sm;
    return PBE_OK;
}

pbe_status pbe_batch_steps(pbe_batch* b, int64_t* steps)
{
    if (!b || !steps) return bfail(PBE_EINVAL, "null argument");
    for (int i = 0; i < b->count; ++i) steps[i] = b->h_steps[i];
    return PBE_OK;
}

// The descriptors of the closure instances point at the batch's weights and box.
static pbe_status upload_inst(pbe_batch* b)
{
    BTRY(cudaStreamSynchronize(b->stream));
    BTRY(cudaMemcpy(b->d_inst, b->h_inst.data(), sizeof(BatchInst) * b->count, cudaMemcpyHostToDevice));
    return PBE_OK;
}

pbe_status pbe_batch_set_closure(pbe_batch* b, const float* w, int count)
{
    if (!b || !w) return bfail(PBE_EINVAL, "null argument");
    if (count != kMlpNW) return bfail(PBE_EINVAL, "the closure has %d weights (got %d)", kMlpNW, count);
    for (int k = 0; k < count; ++k)
        if (!std::isfinite(w[k])) return bfail(PBE_EINVAL, "non-finite closure weight %d", k);
    std::vector<__nv_bfloat16> hw;
    std::vector<float> hb;
    pack_closure(w, hw, hb);
    BTRY(cudaStreamSynchronize(b->stream));
    if (!b->d_mW) {
        if (cudaMalloc(&b->d_mW, sizeof(__nv_bfloat16) * hw.size()) != cudaSuccess ||
            cudaMalloc(&b->d_mB, sizeof(float) * hb.size()) != cudaSuccess) {
            cudaGetLastError();
            return bfail(PBE_ENOMEM, "allocating the closure weights failed");
        }
    }
    BTRY(cudaMemcpy(b->d_mW, hw.data(), sizeof(__nv_bfloat16) * hw.size(), cudaMemcpyHostToDevice));
    BTRY(cudaMemcpy(b->d_mB, hb.data(), sizeof(float) * hb.size(), cudaMemcpyHostToDevice));
    for (BatchInst& d : b->h_inst) {
        d.K.mW = b->d_mW;
        d.K.mB = b->d_mB;
    }
    pbe_status st = upload_inst(b);
    if (st) return st;
    b->closure_set = 1;
    return PBE_OK;
}

pbe_status pbe_batch_set_closure_box(pbe_batch* b, const double* lo, const double* hi)
{
    if (!b) return bfail(PBE_EINVAL, "null batch");
    const bool box = lo && hi;   // either bound NULL: no box (as pbe_set_closure_box)
    if (box)
        for (int k = 0; k < 3; ++k)
            if (std::isnan(lo[k]) || std::isnan(hi[k]) || !(lo[k] <= hi[k]))
                return bfail(PBE_EINVAL, "closure box: lo[%d] <= hi[%d] required", k, k);
    for (BatchInst& d : b->h_inst) {
        d.K.mbox = box ? 1 : 0;
        for (int k = 0; k < 3; ++k) {
            d.K.mlo[k] = box ? lo[k] : 0.0;
            d.K.mhi[k] = box ? hi[k] : 0.0;
        }
    }
    return upload_inst(b);
}

pbe_status pbe_batch_set_schedule(pbe_batch* b, int warps_per_block, int team_instances, int warp_cells)
{
    if (!b) return bfail(PBE_EINVAL, "null batch");
    if (!batch_kernel(warps_per_block)) return bfail(PBE_EINVAL, "warps_per_block must be 1, 2, 3, 4, 6 or 8");
    if (team_instances < 0 || team_instances > b->count)
        return bfail(PBE_EINVAL, "team_instances = %d outside [0, %d]", team_instances, b->count);
    if (warp_cells < 0 || warp_cells > kMaxBatchCells)
        return bfail(PBE_EINVAL, "warp_cells = %d outside [0, %d]", warp_cells, kMaxBatchCells);
    if (!schedule_fits(b, warps_per_block, team_instances, warp_cells))
        return bfail(PBE_EINVAL,
                     "%d warps a block with %d team instances and warp instances of up to %d cells do not fit in "
                     "one block's shared memory",
                     warps_per_block, team_instances, warp_cells);
    BTRY(upload_order(b, team_instances, warp_cells));
    b->wpb = warps_per_block;
    b->nteam = team_instances;
    b->wcells = warp_cells;
    return PBE_OK;
}

pbe_status pbe_batch_get_schedule(pbe_batch* b, int* warps_per_block, int* team_instances, int* warp_cells)
{
    if (!b) return bfail(PBE_EINVAL, "null batch");
    if (warps_per_block) *warps_per_block = b->wpb;
    if (team_instances) *team_instances = b->nteam;
    if (warp_cells) *warp_cells = b->wcells;
    return PBE_OK;
}

pbe_status pbe_batch_set_config(pbe_batch* b, int warps_per_block)
{
    if (!b) return bfail(PBE_EINVAL, "null batch");
    return pbe_batch_set_schedule(b, warps_per_block, 0, kMaxBatchCells);
}

pbe_status pbe_batch_solve(pbe_batch* b, const double* t_out, int n_out, double* rows, int mem, int64_t* total_steps)
{
    if (!b || !rows) return bfail(PBE_EINVAL, "null argument");
    if (b->mlp && !b->closure_set)
        return bfail(PBE_ESTATE, "instances with the learned closure: set its weights first (pbe_batch_set_closure)");
    pbe_status st = check_times(b, t_out, n_out);
    if (st) return st;
    for (int i = 0; i < b->count; ++i)
        if (t_out[0] < b->t0[i]) return bfail(PBE_EINVAL, "t_out[0] precedes instance %d's start time", i);
    st = ensure_tout(b, n_out);
    if (st) return st;
    BTRY(cudaMemcpyAsync(b->d_tout, t_out, sizeof(double) * n_out, cudaMemcpyHostToDevice, b->stream));
    st = run_batch(b, n_out);
    if (st) return st;
    cudaMemcpyKind kd = mem == PBE_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    BTRY(cudaMemcpyAsync(rows, b->d_rows, sizeof(double) * 6 * (size_t)n_out * b->count, kd, b->stream));
    return collect_status(b, total_steps);
}

pbe_status pbe_batch_autotune(pbe_batch* b, const double* t_out, int n_out, int* chosen)
{
    if (!b) return bfail(PBE_EINVAL, "null batch");
    if (b->mlp && !b->closure_set)
        return bfail(PBE_ESTATE, "instances with the learned closure: set its weights first (pbe_batch_set_closure)");
    pbe_status st = check_times(b, t_out, n_out);
    if (st) return st;
    st = ensure_tout(b, n_out);
    if (st) return st;
    // keep the state: every trial restarts from it
    double *save = nullptr, *saveC = nullptr, *savet = nullptr;
    if (cudaMalloc(&save, sizeof(double) * b->total_cells) != cudaSuccess ||
        cudaMalloc(&saveC, sizeof(double) * b->count) != cudaSuccess ||
        cudaMalloc(&savet, sizeof(double) * b->count) != cudaSuccess) {
        cudaFree(save); cudaFree(saveC); cudaFree(savet);
        return bfail(PBE_ENOMEM, "autotune scratch allocation failed");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best = 1e30f;
    int best_w = b->wpb, best_t = b->nteam, best_c = b->wcells;
    // the trials; every exit path below frees the scratch and events
    auto run = [&]() -> pbe_status {
        BTRY(cudaMemcpyAsync(save, b->d_state, sizeof(double) * b->total_cells, cudaMemcpyDeviceToDevice, b->stream));
        BTRY(cudaMemcpyAsync(saveC, b->d_C, sizeof(double) * b->count, cudaMemcpyDeviceToDevice, b->stream));
        BTRY(cudaMemcpyAsync(savet, b->d_t, sizeof(double) * b->count, cudaMemcpyDeviceToDevice, b->stream));
        BTRY(cudaMemcpyAsync(b->d_tout, t_out, sizeof(double) * n_out, cudaMemcpyHostToDevice, b->stream));
        BTRY(cudaEventCreate(&e0));
        BTRY(cudaEventCreate(&e1));
        // time one schedule (the first of two runs warms up); <0 when it does not fit
        auto trial = [&](int w, int nt, int wc, float* ms_out) -> cudaError_t {
            *ms_out = -1.0f;
            if (!schedule_fits(b, w, nt, wc)) return cudaSuccess;
            cudaError_t e = upload_order(b, nt, wc);
            if (e != cudaSuccess) return e;
            float ms = 0.0f;
            for (int rep = 0; rep < 2; ++rep) {
                if ((e = cudaMemcpyAsync(b->d_state, save, sizeof(double) * b->total_cells, cudaMemcpyDeviceToDevice,
                                         b->stream)) != cudaSuccess ||
                    (e = cudaMemcpyAsync(b->d_C, saveC, sizeof(double) * b->count, cudaMemcpyDeviceToDevice,
                                         b->stream)) != cudaSuccess ||
                    (e = cudaMemcpyAsync(b->d_t, savet, sizeof(double) * b->count, cudaMemcpyDeviceToDevice,
                                         b->stream)) != cudaSuccess ||
                    (e = cudaEventRecord(e0, b->stream)) != cudaSuccess ||
                    (e = launch_batch(b, w, nt, wc, n_out, b->stream)) != cudaSuccess ||
                    (e = cudaEventRecord(e1, b->stream)) != cudaSuccess ||
                    (e = cudaEventSynchronize(e1)) != cudaSuccess || (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
                    return e;
            }
            *ms_out = ms;
            return cudaSuccess;
        };
        std::set<std::tuple<int, int, int>> tried;
        auto consider = [&](int w, int nt, int wc) -> cudaError_t {
            if (nt < 0 || nt > b->count || wc < 0 || !tried.insert({w, nt, wc}).second) return cudaSuccess;
            float ms;
            cudaError_t e = trial(w, nt, wc, &ms);
            if (e == cudaSuccess && ms >= 0.0f && ms < best) { best = ms; best_w = w; best_t = nt; best_c = wc; }
            return e;
        };
        // (1) every warps-per-block setting with 0, d/2, d and 2d of the
        // costliest instances as teams (d: the cost heuristic's count), with
        // the largest size cut that fits ...
        const int d = b->nteam_default;
        const int cands[] = {1, 2, 3, 4, 6, 8};
        for (int w : cands)
            for (int nt : {0, d / 2, d, 2 * d}) BTRY(consider(w, nt, fitting_wcells(b, w, nt, kMaxBatchCells)));
        // (2) ... then, at the fastest, the largest size cut of every higher
        // occupancy level (the warp slices shrink as the size cut falls) ...
        {
            const int w = best_w, nt = best_t;
            int level = blocks_per_sm(b, w, nt, best_c);
            std::vector<int> cuts(b->sizes_desc);
            cuts.push_back(0);
            for (int N : cuts) {
                if (N >= best_c || !schedule_fits(b, w, nt, N)) continue;
                const int k = blocks_per_sm(b, w, nt, N);
                if (k > level) {
                    level = k;
                    BTRY(consider(w, nt, N));
                }
            }
        }
        // (3) ... and team counts around the fastest
        {
            const int w = best_w, t = best_t, c = best_c;
            for (int nt : {t / 4, t / 2, (3 * t) / 4, (5 * t) / 4, (3 * t) / 2, 2 * t, 3 * t})
                BTRY(consider(w, nt, fitting_wcells(b, w, std::min(nt, b->count), c)));
        }
        BTRY(upload_order(b, best_t, best_c));
        BTRY(cudaMemcpyAsync(b->d_state, save, sizeof(double) * b->total_cells, cudaMemcpyDeviceToDevice, b->stream));
        BTRY(cudaMemcpyAsync(b->d_C, saveC, sizeof(double) * b->count, cudaMemcpyDeviceToDevice, b->stream));
        BTRY(cudaMemcpyAsync(b->d_t, savet, sizeof(double) * b->count, cudaMemcpyDeviceToDevice, b->stream));
        BTRY(cudaStreamSynchronize(b->stream));
        return PBE_OK;
    };
    st = run();
    cudaStreamSynchronize(b->stream);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(save); cudaFree(saveC); cudaFree(savet);
    if (st) return st;
    b->wpb = best_w;
    b->nteam = best_t;
    b->wcells = best_c;
    if (chosen) *chosen = best_w;
    return PBE_OK;
}

}  // extern "C"

// Batched discrete adjoint of 1-D instances: a team of W warps (one block)
// differentiates one instance at a time (forward with checkpoints every K
// steps, then the reverse sweep segment by segment with recomputation),
// keeping the state, the adjoint vectors and the face coefficients in the
// block's shared memory.  Same reverse-mode arithmetic as the persistent
// single-grid adjoint (the fast forward's face derivative, flat below
// 2^-959; step length through its CFL or clip branch; pending moment-weight
// terms added on the fly; rate adjoints from the recorded rates and ln s,
// kin_backward).  The warps share the rows of the forward stages and the faces and
// cells of the reverse ones; sums are warp butterflies combined in warp order
// through shared memory, and the scalar chain is replicated in every lane.
// W is chosen on the host from the batch size (enough warps for every SM).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "pbe_adjoint.cuh"
#include "pbe_chain.cuh"
#include "pbe_internal.h"
#include "pbe_tiles.cuh"

void pbe_set_error_message(int code, const char* msg);  // pbe_api.cu

namespace pbe {

__host__ __device__ inline int badj_np(int N) { return 32 * ((N + 31) / 32 + 1) + 3; }

// scalar record of one step: state at its start and the chain values
struct StepRec1 {
    double C, t, V0, dt, t_new, G1a, Ba, La, C1, G1b, Bb, Lb;   // La, Lb: ln s at the two stages
    int clipped, out_idx;
};

__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Pairwise sum of n values (a fixed tree: the same on every run).
template <int N>
__device__ __forceinline__ double tree_sum(const double* p)
{
    if constexpr (N == 1) return p[0];
    else return tree_sum<N / 2>(p) + tree_sum<N - N / 2>(p + N / 2);
}

// Block-level sums of a team of W warps: warp butterflies, then the warp
// sums added pairwise in a fixed tree (two buffers used alternately so that
// one barrier per sum suffices; the barrier also orders the shared-memory
// writes before the sum against the reads after it).  W = 1: the butterfly
// alone.
template <int W>
struct Team {
    double* red;   // [2][W] in shared memory
    int par;
    __device__ __forceinline__ void sync() const
    {
        if (W == 1) __syncwarp();
        else __syncthreads();
    }
    __device__ __forceinline__ double sum(double v)
    {
        v = wsum(v);
        if (W == 1) {
            __syncwarp();
            return v;
        }
        if ((threadIdx.x & 31) == 0) red[par * W + (threadIdx.x >> 5)] = v;
        __syncthreads();
        const double t = tree_sum<W>(red + par * W);
        par ^= 1;
        return t;
    }
};

// forward stage over the rows [r0, r1) of this warp (fused-path quotient),
// as in pbe_batch.cu; returns this lane's partial of the volume moment.  The
// weights x_i^3 dL = (2i+1)^3 (dL/2)^3 dL: the integer cube exactly (i below
// 2^17), the factor once at the end.
template <int STAGE>
__device__ __forceinline__ double fwd_stage(const double* in, const double* old, double* out, int N, int r0, int r1,
                                            double c1, double src, double d1)
{
    const int lane = threadIdx.x & 31;
    double hcur = face_value<true>(in[32 * r0 + lane], in[32 * r0 + lane + 1], in[32 * r0 + lane + 2]);
    double m3 = 0.0;
    for (int r = r0; r < r1; ++r) {
        const int fn = 32 * (r + 1) + lane;
        const double hnext = face_value<true>(in[fn], in[fn + 1], in[fn + 2]);
        const double a = __shfl_down_sync(0xffffffffu, hcur, 1);
        const double b = __shfl_sync(0xffffffffu, hnext, 0);
        const double hright = lane == 31 ? b : a;
        const int i = 32 * r + lane;
        if (i < N) {
            double v = in[i + 2] + c1 * (hcur - hright);
            if (i == 0) v += src;
            if (STAGE == 2) v = 0.5 * old[i + 2] + 0.5 * v;
            out[i + 2] = v;
            const long long w1 = 2LL * i + 1;
            m3 = fma(exact_int_double(w1 * w1 * w1), v, m3);
        }
        hcur = hnext;
    }
    const double hd = 0.5 * d1;
    return m3 * (((hd * hd) * hd) * d1);
}

// adjoint of one stage by the team.  nt: stage input (cell i at [i+2]);
// lam: adjoint of the stage output (cell i at [i+2]) to which pending(p)
// is added (p = moment-weight coefficients, scale s: lam_eff = s (lam + p.W));
// writes lam_eff into leff[i+2] and the three derivative coefficients of
// every face f into jt[3f..3f+2] (to cells f-2, f-1, f).  Returns
// dot = lam_eff . D(n) and l0 = lam_eff at cell 0.
template <int W>
__device__ __forceinline__ void adj_stage(const double* nt, const double* lam, const double* p, double s, double* leff,
                                          double* jt, int N, int R, double d1, Team<W>& tm, double& dot, double& l0)
{
    constexpr int NT = 32 * W;
    const int tid = threadIdx.x;
    const double invd = 1.0 / d1;   // once per stage
    // effective lambda with zero ghosts; the pending weights sum_k p_k x^k dL
    // as a polynomial in the exact integer 2i+1 (x = (2i+1) dL/2), its
    // coefficients p_k (dL/2)^k dL formed once per stage
    const double hd = 0.5 * d1, q0 = p[0] * d1, q1 = p[1] * (hd * d1), q2 = p[2] * ((hd * hd) * d1),
                 q3 = p[3] * (((hd * hd) * hd) * d1);
    for (int k = tid; k < 32 * (R + 1) + 3; k += NT) {
        const int i = k - 2;
        double v = 0.0;
        if (i >= 0 && i < N) {
            const double w = exact_int_double(2LL * i + 1);
            v = s * (lam[k] + (q0 + w * (q1 + w * (q2 + w * q3))));
        }
        leff[k] = v;
    }
    tm.sync();
    // faces f = 0..32(R+1)-1; coefficient of face f into cells f-2, f-1, f
    double acc = 0.0;
    for (int k = tid; k < 32 * (R + 1); k += NT) {
        const int f = k;
        FaceAdj fa{0.0, 0.0, 0.0, 0.0};
        if (f <= N) {   // the forward's fast face (flat below 2^-959); mu = (lam_f - lam_{f-1}) / dL
            fa = face_adj_fast(nt[f], nt[f + 1], nt[f + 2], leff[f + 1], leff[f + 2], invd);
            acc += fa.hmu;
        }
        jt[3 * k] = fa.cm2;
        jt[3 * k + 1] = fa.cm1;
        jt[3 * k + 2] = fa.c0;
    }
    dot = tm.sum(acc);   // its barrier also orders the jt writes before their reads
    l0 = leff[2];
}

// One instance at a time per block of W warps (the team); slot = the
// block's scratch in the checkpoint and segment stores.  The forward pass
// also records the steps of the segment it is in (the last segment is then
// not recomputed).
template <int W>
__global__ void __launch_bounds__(W * 32) k_batch_vjp(const BatchInst* __restrict__ inst, const int* __restrict__ order,
                                                      int count, const double* __restrict__ state0,
                                                      const double* __restrict__ C0s, const double* __restrict__ t0s,
                                                      const double* __restrict__ t_out, int n_out,
                                                      const double* __restrict__ seeds, int K, int max_ckpt,
                                                      double* ckpt, StepRec1* ckrec, double* segn, double* segn1,
                                                      StepRec1* segrec, double* dth_out, double* dn0_out,
                                                      int* status_out, unsigned int* queue, int np_max)
{
    constexpr int NT = 32 * W;
    extern __shared__ double smem[];
    __shared__ double red[2 * W];
    __shared__ double chs[6];   // chain values handed from warp 0 to the team
    __shared__ RateCarry rcs[32];   // warp 0: a step's stage-2 evaluation, for the next step's rates (the same time)
    __shared__ double pcs[4], pus[4];   // pending moment-weight coefficients of the stage adjoints
    __shared__ int s_idx;
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long slot = blockIdx.x;
    Team<W> tm{red, 0};
    // arrays of np_max: nb, n1b, lam, lamo, u, faces (3 per face), leff
    double* nb = smem;
    double* n1b = nb + np_max;
    double* lam = n1b + np_max;
    double* lamo = lam + np_max;
    double* u = lamo + np_max;
    double* fc = u + np_max;     // 3 * np_max
    double* leff = fc + 3 * np_max;
    double* my_ck = ckpt + slot * (long long)max_ckpt * np_max;
    StepRec1* my_ckr = ckrec + slot * max_ckpt;
    double* my_sn = segn + slot * (long long)K * np_max;
    double* my_sn1 = segn1 + slot * (long long)K * np_max;
    StepRec1* my_sr = segrec + slot * K;
    for (;;) {
        if (tid == 0) s_idx = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= count) break;
        const int id = order[idx];
        const Kin Kn = inst[id].K;
        const Geom g = inst[id].g;
        const long long off = inst[id].offset;
        const int N = g.N1, R = inst[id].rows;
        const int r0 = (warp * R) / W, r1 = ((warp + 1) * R) / W;   // this warp's rows in the forward stages
        const int np = badj_np(N);
        const double d1 = g.d1;
        const double* sd = seeds + (size_t)id * n_out * 6;
        int status = 0;
        lam = n1b + np_max;
        lamo = lam + np_max;
        for (int k = tid; k < np; k += NT) {
            const int i = k - 2;
            nb[k] = (i >= 0 && i < N) ? state0[off + i] : 0.0;
            n1b[k] = 0.0;
        }
        tm.sync();
        // ---------------- forward with checkpoints ----------------
        StepRec1 s;
        s.C = C0s[id];
        s.t = t0s[id];
        {
            double m3 = 0.0;   // the volume moment with fwd_stage's weights
            for (int i = tid; i < N; i += NT) {
                const long long w1 = 2LL * i + 1;
                m3 = fma(exact_int_double(w1 * w1 * w1), nb[i + 2], m3);
            }
            const double hd = 0.5 * d1;
            s.V0 = tm.sum(m3 * (((hd * hd) * hd) * d1));
        }
        int out_idx = 0;
        // the chain's last stage-2 evaluation (time and solubility) for the series
        double rct = __longlong_as_double(0x7ff8000000000000LL), rccs = 0.0;
        if (W == 1 || warp == 0) rate_carry_init(rcs[tid & 31], Kn);
        const bool row0 = n_out > 0 && t_out[0] == s.t;
        while (out_idx < n_out && t_out[out_idx] == s.t) ++out_idx;
        long long total = 0;
        bool done = out_idx >= n_out;
        // The chain's rates and step length: computed by warp 0 alone in a team
        // and handed to the others through shared memory (the team waits for
        // them either way; the other warps' FP64 pipe time goes to cells).
        auto prepare = [&](StepRec1& r) {
            double G1, G2, B, dt, tn, L;
            int clipped = 0;
            if (W == 1 || warp == 0) {
                // at the time of the last stage-2 evaluation: the series from it
                if (!(r.t == rct && rates_by_series(rcs[tid & 31], r.C, rccs, 1, G1, G2, B, L)))
                    kinetics_warp<false>(Kn, r.C, r.t, G1, G2, B, &L);
                clipped = timestep_fast(Kn, g, G1, G2, r.t, t_out[out_idx], dt, tn);
            }
            if (W > 1) {
                if (tid == 0) {
                    chs[0] = G1; chs[1] = B; chs[2] = L; chs[3] = dt; chs[4] = tn; chs[5] = clipped;
                }
                __syncthreads();
                G1 = chs[0]; B = chs[1]; L = chs[2]; dt = chs[3]; tn = chs[4]; clipped = (int)chs[5];
            }
            r.G1a = G1; r.Ba = B; r.La = L; r.dt = dt; r.t_new = tn; r.out_idx = out_idx; r.clipped = clipped;
        };
        auto stage2_rates = [&](StepRec1& r) {
            double G1, G2, B, L;
            if (W == 1 || warp == 0) {
                const KinT tc = kin_temperature(Kn, r.t_new);
                double rec[2];
                kinetics_warp_T<false>(Kn, r.C1, tc, G1, G2, B, &L, nullptr, rec);
                rate_carry_keep(rcs[tid & 31], Kn, G1, G2, B, L, rec);
                rct = r.t_new;
                rccs = tc.cs;
            }
            if (W > 1) {
                if (tid == 0) { chs[0] = G1; chs[1] = B; chs[2] = L; }
                __syncthreads();
                G1 = chs[0]; B = chs[1]; L = chs[2];
            }
            r.G1b = G1; r.Bb = B; r.Lb = L;
        };
        const double inv_cfl = 1.0 / Kn.cfl;
        // 1/kg1 and 1/kb (0 when the prefactor is 0) for the rate adjoints
        const double ik[3] = {Kn.kg1 > 0.0 ? 1.0 / Kn.kg1 : 0.0, 0.0, Kn.kb > 0.0 ? 1.0 / Kn.kb : 0.0};
        // one step from record r (state in nb); fills C1, G1b, Bb; advances r to the next step's start
        auto step = [&](StepRec1& r, bool record, long long q) {
            if (record) {
                for (int k = tid; k < np; k += NT) my_sn[q * np_max + k] = nb[k];
            }
            const double V1 =
                tm.sum(fwd_stage<1>(nb, nb, n1b, N, r0, r1, r.G1a * r.dt * g.inv_d1, r.dt * r.Ba * g.inv_d1, d1));
            r.C1 = r.C - Kn.kappa * (V1 - r.V0);
            stage2_rates(r);
            if (record) {
                for (int k = tid; k < np; k += NT) my_sn1[q * np_max + k] = n1b[k];
                if (tid == 0) my_sr[q] = r;
            }
            const double V2 =
                tm.sum(fwd_stage<2>(n1b, nb, nb, N, r0, r1, r.G1b * r.dt * g.inv_d1, r.dt * r.Bb * g.inv_d1, d1));
            StepRec1 nx = r;
            nx.C = r.C - Kn.kappa * (V2 - r.V0);
            nx.t = r.t_new;
            nx.V0 = V2;
            if (r.clipped) out_idx = r.out_idx + 1;
            r = nx;
        };
        if (!done) prepare(s);
        while (!done) {
            if (total % K == 0) {
                const long long c = total / K;
                if (c >= max_ckpt) { status = PBE_ETIMEOUT; break; }
                for (int k = tid; k < np; k += NT) my_ck[c * np_max + k] = nb[k];
                if (tid == 0) my_ckr[c] = s;
            }
            step(s, true, total % K);
            ++total;
            if (!isfinite(s.C) || !isfinite(s.V0)) { status = PBE_ENONFINITE; break; }
            if (out_idx >= n_out) done = true;
            else prepare(s);
        }
        tm.sync();
        // ---------------- reverse sweep ----------------
        // The scalar adjoint chain (seed rows, solute balance, rate adjoints,
        // step length) runs in warp 0 alone; the team needs only the pending
        // moment-weight coefficients of each stage adjoint, handed over in
        // pcs / pus (shared memory) before the barrier that precedes the stage.
        const bool chain = W == 1 || warp == 0;
        double lC = 0.0, lt = 0.0, lth[6] = {0, 0, 0, 0, 0, 0};
        double pc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k = tid; k < np; k += NT) lam[k] = 0.0;
        tm.sync();
        const long long nck = status ? 0 : (total + K - 1) / K;
        for (long long c = nck - 1; c >= 0; --c) {
            const long long s0 = c * K, s1 = (s0 + K < total) ? s0 + K : total;
            if (c < nck - 1) {   // the last segment's records come from the forward pass
                for (int k = tid; k < np; k += NT) {
                    nb[k] = my_ck[c * np_max + k];
                    n1b[k] = 0.0;
                }
                tm.sync();
                StepRec1 r = my_ckr[c];
                out_idx = r.out_idx;
                for (long long q = 0; q < s1 - s0; ++q) {
                    if (q > 0) prepare(r);
                    step(r, true, q);
                }
            }
            tm.sync();
            for (long long q = s1 - s0 - 1; q >= 0; --q) {
                const StepRec1 rr = my_sr[q];
                double lV0 = 0.0, lCprev = 0.0;
                if (chain) {
                    if (rr.clipped) {
                        const double* row = sd + (size_t)rr.out_idx * 6;
                        for (int k = 0; k < 4; ++k) pc[k] += row[1 + k];
                        lC += row[5];
                    }
                    lV0 = Kn.kappa * lC;
                    lCprev = lC;
                    pc[3] += -Kn.kappa * lC;
                    if (tid == 0)
                        for (int k = 0; k < 4; ++k) pcs[k] = pc[k];
                }
                // stage-2 adjoint: input n1 (recorded), lam_eff = (lam + pc.W)/2
                for (int k = tid; k < np; k += NT) nb[k] = my_sn1[q * np_max + k];
                tm.sync();
                double P1, P0;
                adj_stage<W>(nb, lam, pcs, 0.5, leff, fc, N, R, d1, tm, P1, P0);
                for (int i = tid; i < N; i += NT) {
                    const double jt = fc[3 * (i + 2)] + fc[3 * (i + 1) + 1] + fc[3 * i + 2];
                    const double l2 = leff[i + 2];
                    lamo[i + 2] = l2;
                    u[i + 2] = l2 + rr.dt * rr.G1b * jt;
                }
                double ldt = 0.0, ltn = 0.0;
                if (chain) {
                    ldt = rr.G1b * P1 + rr.Bb * P0 * g.inv_d1;
                    double lC1 = 0.0;
                    ltn = lt;
                    kin_backward(Kn, ik, rr.C1, rr.t_new, rr.G1b, 0.0, rr.Bb, rr.Lb, 0.0, 0.0, rr.dt * P1, 0.0,
                                 rr.dt * P0 * g.inv_d1, &lC1, &ltn, lth);
                    lCprev += lC1;
                    lV0 += Kn.kappa * lC1;
                    if (tid == 0) {
                        pus[0] = 0.0; pus[1] = 0.0; pus[2] = 0.0;
                        pus[3] = -Kn.kappa * lC1;
                    }
                }
                // stage-1 adjoint: input n (recorded), lam_eff = u + pu.W
                tm.sync();   // nb, leff and fc are rewritten below; pus is complete
                for (int k = tid; k < np; k += NT) nb[k] = my_sn[q * np_max + k];
                tm.sync();
                adj_stage<W>(nb, u, pus, 1.0, leff, fc, N, R, d1, tm, P1, P0);
                for (int i = tid; i < N; i += NT) {
                    const double jt = fc[3 * (i + 2)] + fc[3 * (i + 1) + 1] + fc[3 * i + 2];
                    lamo[i + 2] += leff[i + 2] + rr.dt * rr.G1a * jt;
                }
                tm.sync();   // lamo complete before it becomes lam; fc, leff free again
                if (chain) {
                    ldt += rr.G1a * P1 + rr.Ba * P0 * g.inv_d1;
                    double lG1 = rr.dt * P1;
                    const double lB = rr.dt * P0 * g.inv_d1;
                    double ltp;
                    if (!rr.clipped) {
                        ltp = ltn;
                        ldt += ltn;
                        // dt = cfl / (G1 / dL): d dt / d G1 = -cfl dL / G1^2 = -dt^2 / (cfl dL)
                        lG1 += -(rr.dt * rr.dt * inv_cfl) * ldt * g.inv_d1;
                    } else {
                        ltp = -ldt;
                    }
                    kin_backward(Kn, ik, rr.C, rr.t, rr.G1a, 0.0, rr.Ba, rr.La, 0.0, 0.0, lG1, 0.0, lB, &lCprev,
                                 &ltp, lth);
                    lC = lCprev;
                    lt = ltp;
                    pc[0] = pc[1] = pc[2] = 0.0;
                    pc[3] = lV0;
                }
                double* tmp = lam;
                lam = lamo;
                lamo = tmp;
            }
        }
        if (chain) {
            if (row0) {
                for (int k = 0; k < 4; ++k) pc[k] += sd[1 + k];
                lC += sd[5];
            }
            if (tid == 0)
                for (int k = 0; k < 4; ++k) pcs[k] = pc[k];
        }
        tm.sync();
        if (dn0_out) {
            for (int i = tid; i < N; i += NT) {
                const double x = (i + 0.5) * d1;
                dn0_out[off + i] = lam[i + 2] + (pcs[0] + x * (pcs[1] + x * (pcs[2] + x * pcs[3]))) * d1;
            }
        }
        if (tid == 0) {
            for (int k = 0; k < 6; ++k) dth_out[(size_t)id * 7 + k] = lth[k];
            dth_out[(size_t)id * 7 + 6] = lC;
            status_out[id] = status;
        }
        __syncthreads();
    }
}

}  // namespace pbe

using namespace pbe;

struct pbe_batch;   // defined in pbe_batch.cu
extern "C" int pbe_batch_internal_vjp_warps(const pbe_batch* b);
extern "C" int pbe_batch_internal_vjp_blocks(const pbe_batch* b);
extern "C" int pbe_batch_internal_power_law(const pbe_batch* b);
extern "C" void** pbe_batch_internal_vjp_work(pbe_batch* b);
extern "C" pbe_status pbe_batch_internal_view(pbe_batch* b, const void** inst, const int** order, int* count,
                                              double** state, double** C, double** t, int* np_max, int* device,
                                              void** stream);

namespace {
pbe_status bafail(pbe_status code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    pbe_set_error_message(code, buf);
    return code;
}

// Device scratch of pbe_batch_vjp, kept with the batch between calls and
// grown when a call needs more (every call ends synchronized, so no launch
// uses a buffer when it is replaced).
struct VjpWork {
    double *ck = nullptr, *sn = nullptr, *sn1 = nullptr, *seeds = nullptr, *dth = nullptr, *tout = nullptr;
    StepRec1 *ckr = nullptr, *sr = nullptr;
    int* status = nullptr;
    unsigned int* queue = nullptr;
    size_t ck_cap = 0, sn_cap = 0, sn1_cap = 0, seeds_cap = 0, dth_cap = 0, tout_cap = 0, ckr_cap = 0, sr_cap = 0,
           status_cap = 0, queue_cap = 0;
    std::vector<double> h_dth;
    std::vector<int> h_status;
};

template <class T>
cudaError_t grow(T*& p, size_t& cap, size_t n)
{
    if (n <= cap) return cudaSuccess;
    cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, sizeof(T) * n);
    if (e == cudaSuccess) cap = n;
    return e;
}
}  // namespace

extern "C" void pbe_batch_internal_free_vjp_work(void* w)
{
    VjpWork* v = (VjpWork*)w;
    if (!v) return;
    cudaFree(v->ck); cudaFree(v->sn); cudaFree(v->sn1); cudaFree(v->seeds); cudaFree(v->dth); cudaFree(v->tout);
    cudaFree(v->ckr); cudaFree(v->sr); cudaFree(v->status); cudaFree(v->queue);
    delete v;
}

#define BATRY(call)                                                                                    \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) { rc = bafail(PBE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); goto out; } \
    } while (0)

extern "C" pbe_status pbe_batch_vjp(pbe_batch* b, const double* t_out, int n_out, const double* seeds_in, int seeds_mem,
                                    int checkpoint_every, double* dL_dtheta, double* dL_dC0, double* dL_dn0, int mem)
{
    const void* inst_v;
    const int* order;
    int count, np_max, device;
    double *state, *Cs, *ts;
    void* stream_v;
    if (!b || !t_out || !seeds_in || !dL_dtheta) return bafail(PBE_EINVAL, "null argument");
    if (dL_dn0 && mem != PBE_MEM_DEVICE) return bafail(PBE_EINVAL, "dL_dn0 must be device memory");
    if (n_out < 1 || checkpoint_every < 1) return bafail(PBE_EINVAL, "n_out and checkpoint_every must be >= 1");
    for (int j = 1; j < n_out; ++j)
        if (!(t_out[j] > t_out[j - 1])) return bafail(PBE_EINVAL, "t_out must increase");
    // the batched adjoint differentiates the power-law form
    if (!pbe_batch_internal_power_law(b))
        return bafail(PBE_EINVAL, "the batched adjoint needs power-law kinetics with the polynomial solubility");
    pbe_batch_internal_view(b, &inst_v, &order, &count, &state, &Cs, &ts, &np_max, &device, &stream_v);
    void** wslot = pbe_batch_internal_vjp_work(b);
    if (!*wslot) *wslot = new VjpWork();
    VjpWork& w = *(VjpWork*)*wslot;
    cudaStream_t st = (cudaStream_t)stream_v;
    const BatchInst* inst = (const BatchInst*)inst_v;
    const int K = checkpoint_every;
    const int max_ckpt = (4096 + K - 1) / K;   // up to 4096 steps per instance
    const int npa = np_max;   // per-instance buffer length (same layout as the forward batch)
    pbe_status rc = PBE_OK;
    int W = pbe_batch_internal_vjp_warps(b), occ = 0, sms = 0, maxsm = 0;
    size_t smem = 0;
    long long slots = 0;
    const void* fn = nullptr;
    BATRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    BATRY(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    if (count < 1) goto out;
    // warps per instance (measured on the 500-cell gradient workload: teams of
    // 4 while there are at most 8 instances per SM, else of 2)
    if (W == 0) W = (long long)count <= 8LL * sms ? 4 : 2;
    smem = (size_t)10 * npa * sizeof(double);
    if (smem + 2 * 8 * sizeof(double) + 64 > (size_t)maxsm) {
        rc = bafail(PBE_EINVAL, "instances too large for the batched adjoint");
        goto out;
    }
    fn = W == 8 ? (const void*)k_batch_vjp<8>
       : W == 4 ? (const void*)k_batch_vjp<4>
       : W == 2 ? (const void*)k_batch_vjp<2>
                : (const void*)k_batch_vjp<1>;
    BATRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    BATRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, W * 32, smem));
    if (occ < 1) { rc = bafail(PBE_ECUDA, "batched adjoint kernel does not fit on an SM"); goto out; }
    {
        // resident teams per SM: one while there are at most 2 instances per SM
        // (the costliest instances, pulled first, keep an SM to themselves),
        // else 8 warps' worth
        int per_sm = pbe_batch_internal_vjp_blocks(b);
        if (per_sm == 0) per_sm = (long long)count <= 2LL * sms ? 1 : (8 / W > 1 ? 8 / W : 1);
        int blocks = (per_sm < occ ? per_sm : occ) * sms;
        if (blocks > count) blocks = count;
        slots = blocks;
        BATRY(grow(w.ck, w.ck_cap, (size_t)slots * max_ckpt * npa));
        BATRY(grow(w.ckr, w.ckr_cap, (size_t)slots * max_ckpt));
        BATRY(grow(w.sn, w.sn_cap, (size_t)slots * K * npa));
        BATRY(grow(w.sn1, w.sn1_cap, (size_t)slots * K * npa));
        BATRY(grow(w.sr, w.sr_cap, (size_t)slots * K));
        BATRY(grow(w.seeds, w.seeds_cap, (size_t)count * n_out * 6));
        BATRY(grow(w.dth, w.dth_cap, (size_t)count * 7));
        BATRY(grow(w.status, w.status_cap, (size_t)count));
        BATRY(grow(w.queue, w.queue_cap, (size_t)1));
        BATRY(grow(w.tout, w.tout_cap, (size_t)n_out));
        w.h_dth.resize((size_t)count * 7);
        w.h_status.resize(count);
        BATRY(cudaMemcpyAsync(w.seeds, seeds_in, sizeof(double) * (size_t)count * n_out * 6,
                              seeds_mem == PBE_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        BATRY(cudaMemcpyAsync(w.tout, t_out, sizeof(double) * n_out, cudaMemcpyHostToDevice, st));
        BATRY(cudaMemsetAsync(w.queue, 0, sizeof(unsigned int), st));
        double* dn0_dev = (dL_dn0 && mem == PBE_MEM_DEVICE) ? dL_dn0 : nullptr;
        int npa_arg = npa;
        void* args[] = {&inst, &order, &count, &state, &Cs, &ts, &w.tout, &n_out, &w.seeds, (void*)&K,
                        (void*)&max_ckpt, &w.ck, &w.ckr, &w.sn, &w.sn1, &w.sr, &w.dth, &dn0_dev, &w.status,
                        &w.queue, &npa_arg};
        BATRY(cudaLaunchKernel(fn, blocks, W * 32, args, smem, st));
        BATRY(cudaMemcpyAsync(w.h_dth.data(), w.dth, sizeof(double) * (size_t)count * 7, cudaMemcpyDeviceToHost, st));
        BATRY(cudaMemcpyAsync(w.h_status.data(), w.status, sizeof(int) * count, cudaMemcpyDeviceToHost, st));
        BATRY(cudaStreamSynchronize(st));
    }
    for (int i = 0; i < count; ++i) {
        for (int k = 0; k < 6; ++k) dL_dtheta[(size_t)i * 6 + k] = w.h_dth[(size_t)i * 7 + k];
        if (dL_dC0) dL_dC0[i] = w.h_dth[(size_t)i * 7 + 6];
    }
    for (int i = 0; i < count; ++i)
        if (w.h_status[i] != PBE_OK) {
            rc = bafail(w.h_status[i], "instance %d: status %d in the batched adjoint", i, w.h_status[i]);
            break;
        }
out:
    cudaStreamSynchronize(st);
    return rc;
}

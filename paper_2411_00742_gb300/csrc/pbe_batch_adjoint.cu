// Batched discrete adjoint of 1-D instances: one warp differentiates one
// instance at a time (forward with checkpoints every K steps, then the
// reverse sweep segment by segment with recomputation), keeping the state,
// the adjoint vectors and the face coefficients in the warp's slice of shared
// memory.  Same reverse-mode arithmetic as pbe_adjoint.cu (limiter
// derivative of the branch taken, flat below 2^-959; step length through its
// CFL or clip branch; pending moment-weight terms added on the fly), with
// warp butterflies for the reductions and the scalar chain replicated in
// every lane of the warp.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "pbe_internal.h"
#include "pbe_tiles.cuh"

void pbe_set_error_message(int code, const char* msg);  // pbe_api.cu

namespace pbe {

__host__ __device__ inline int badj_np(int N) { return 32 * ((N + 31) / 32 + 1) + 3; }

// scalar record of one step: state at its start and the chain values
struct StepRec1 {
    double C, t, V0, dt, t_new, G1a, Ba, C1, G1b, Bb;
    int clipped, out_idx;
};

__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// forward stage on the warp (fused-path quotient), as in pbe_batch.cu
template <int STAGE>
__device__ __forceinline__ double fwd_stage(const double* in, const double* old, double* out, int N, int R, double c1,
                                            double src, double d1)
{
    const int lane = threadIdx.x & 31;
    double hcur = face_value<true>(in[lane], in[lane + 1], in[lane + 2]);
    double x = (lane + 0.5) * d1, m3 = 0.0;
    for (int r = 0; r < R; ++r) {
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
            m3 += x * x * x * (v * d1);
        }
        hcur = hnext;
        x += 32.0 * d1;
    }
    return wsum(m3);
}

__device__ __forceinline__ void kin_adj(const Kin& K, double C, double t, double lG1, double lB, double* lC, double* lt,
                                        double* lth)
{
    if (K.kind == PBE_KINETICS_FIXED) {
        lth[0] += lG1;
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
    const double ls = pbe_log(s);
    const double s1 = pbe_exp(K.g1 * ls), sb = pbe_exp(K.b * ls);
    const double G1 = K.kg1 * s1, B = K.kb * sb;
    const double lsum = lG1 * K.g1 * G1 / s + lB * K.b * B / s;
    lth[0] += lG1 * s1;
    lth[1] += lG1 * G1 * ls;
    lth[4] += lB * sb;
    lth[5] += lB * B * ls;
    *lC += lsum / cs;
    *lt += lsum * (-C * dcs / (cs * cs)) * dTdt;
}

// adjoint of one stage on the warp.  nt: stage input (cell i at [i+2]);
// lam: adjoint of the stage output (cell i at [i+2]) to which pending(p)
// is added (p = moment-weight coefficients, scale s: lam_eff = s (lam + p.W));
// writes lam_eff into leff[i+2] and the three derivative coefficients of
// every face f into jt[3f..3f+2] (to cells f-2, f-1, f).  Returns
// dot = lam_eff . D(n) and l0 = lam_eff at cell 0.
__device__ __forceinline__ void adj_stage(const double* nt, const double* lam, const double* p, double s, double* leff,
                                          double* jt, int N, int R, double d1, double& dot, double& l0)
{
    const int lane = threadIdx.x & 31;
    const double invd = 1.0 / d1;
    // effective lambda with zero ghosts
    for (int k = lane; k < 32 * (R + 1) + 3; k += 32) {
        const int i = k - 2;
        double v = 0.0;
        if (i >= 0 && i < N) {
            const double x = (i + 0.5) * d1;
            v = s * (lam[k] + (p[0] + x * (p[1] + x * (p[2] + x * p[3]))) * d1);
        }
        leff[k] = v;
    }
    __syncwarp();
    // faces f = 0..32(R+1)-1; coefficient of face f into cells f-2, f-1, f
    double acc = 0.0;
    for (int k = lane; k < 32 * (R + 1); k += 32) {
        const int f = k;
        double cm2 = 0.0, cm1 = 0.0, c0 = 0.0;
        if (f <= N) {
            const double nm2 = nt[f], up = nt[f + 1], dn = nt[f + 2];
            const double a = up - nm2, b = dn - up;
            double pa = 0.0, pb = 0.0, half = 0.0;
            if ((a > 0.0 && b > 0.0) || (a < 0.0 && b < 0.0)) {
                if (fabs(a) >= kPsiFlat && fabs(b) >= kPsiFlat) {
                    const double rs = 1.0 / (a + b), qa = b * rs, qb = a * rs;   // one division per face
                    half = a * qa;
                    pa = 2.0 * qa * qa;
                    pb = 2.0 * qb * qb;
                } else {
                    half = a * (b / (a + b));   // flat tail: the reciprocal of a + b may overflow
                }
            }
            const double mu = (leff[f + 2] - leff[f + 1]) * invd;   // (lam_f - lam_{f-1}) / dL
            cm2 = -0.5 * pa * mu;
            cm1 = (1.0 + 0.5 * (pa - pb)) * mu;
            c0 = 0.5 * pb * mu;
            acc += (up + half) * mu;
        }
        jt[3 * k] = cm2;
        jt[3 * k + 1] = cm1;
        jt[3 * k + 2] = c0;
    }
    __syncwarp();
    dot = wsum(acc);
    l0 = leff[2];
}

template <int WPB>
__global__ void __launch_bounds__(WPB * 32) k_batch_vjp(const BatchInst* __restrict__ inst, const int* __restrict__ order,
                                                        int count, const double* __restrict__ state0,
                                                        const double* __restrict__ C0s, const double* __restrict__ t0s,
                                                        const double* __restrict__ t_out, int n_out,
                                                        const double* __restrict__ seeds, int K, int max_ckpt,
                                                        double* ckpt, StepRec1* ckrec, double* segn, double* segn1,
                                                        StepRec1* segrec, double* dth_out, double* dn0_out,
                                                        int* status_out, unsigned int* queue, int np_max)
{
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long slot = (long long)blockIdx.x * WPB + warp;   // per-warp scratch slot
    // 8 arrays of np_max: nb, n1b, lam, lamo, u, faces (3 * np_max) -- faces need 3 per face
    double* nb = smem + (size_t)warp * 10 * np_max;
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
        int idx = 0;
        if (lane == 0) idx = (int)atomicAdd(queue, 1u);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= count) break;
        const int id = order[idx];
        const Kin Kn = inst[id].K;
        const Geom g = inst[id].g;
        const long long off = inst[id].offset;
        const int N = g.N1, R = inst[id].rows;
        const int np = badj_np(N);
        const double d1 = g.d1;
        const double* sd = seeds + (size_t)id * n_out * 6;
        int status = 0;
        for (int k = lane; k < np; k += 32) {
            const int i = k - 2;
            nb[k] = (i >= 0 && i < N) ? state0[off + i] : 0.0;
            n1b[k] = 0.0;
        }
        __syncwarp();
        // ---------------- forward with checkpoints ----------------
        StepRec1 s;
        s.C = C0s[id];
        s.t = t0s[id];
        {
            double m3 = 0.0, x = (lane + 0.5) * d1;
            for (int i = lane; i < N; i += 32, x += 32.0 * d1) m3 += x * x * x * (nb[i + 2] * d1);
            s.V0 = wsum(m3);
        }
        int out_idx = 0;
        const bool row0 = n_out > 0 && t_out[0] == s.t;
        while (out_idx < n_out && t_out[out_idx] == s.t) ++out_idx;
        long long total = 0;
        bool done = out_idx >= n_out;
        auto prepare = [&](StepRec1& r) {
            double G1, G2, B, dt, tn;
            kinetics_warp<false>(Kn, r.C, r.t, G1, G2, B);
            r.clipped = timestep_fast(Kn, g, G1, G2, r.t, t_out[out_idx], dt, tn);
            r.G1a = G1; r.Ba = B; r.dt = dt; r.t_new = tn; r.out_idx = out_idx;
        };
        // one step from record r (state in nb); fills C1, G1b, Bb; advances r to the next step's start
        auto step = [&](StepRec1& r, bool record, long long q) {
            if (record) {
                for (int k = lane; k < np; k += 32) my_sn[q * np_max + k] = nb[k];
            }
            const double V1 = fwd_stage<1>(nb, nb, n1b, N, R, r.G1a * r.dt / d1, r.dt * r.Ba / d1, d1);
            __syncwarp();
            r.C1 = r.C - Kn.kappa * (V1 - r.V0);
            double G1, G2, B;
            kinetics_warp<false>(Kn, r.C1, r.t_new, G1, G2, B);
            r.G1b = G1; r.Bb = B;
            if (record) {
                for (int k = lane; k < np; k += 32) my_sn1[q * np_max + k] = n1b[k];
                if (lane == 0) my_sr[q] = r;
            }
            const double V2 = fwd_stage<2>(n1b, nb, nb, N, R, r.G1b * r.dt / d1, r.dt * r.Bb / d1, d1);
            __syncwarp();
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
                for (int k = lane; k < np; k += 32) my_ck[c * np_max + k] = nb[k];
                if (lane == 0) my_ckr[c] = s;
                __syncwarp();
            }
            step(s, false, 0);
            ++total;
            if (!isfinite(s.C) || !isfinite(s.V0)) { status = PBE_ENONFINITE; break; }
            if (out_idx >= n_out) done = true;
            else prepare(s);
        }
        // ---------------- reverse sweep ----------------
        double lC = 0.0, lt = 0.0, lth[6] = {0, 0, 0, 0, 0, 0};
        double pc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k = lane; k < np; k += 32) lam[k] = 0.0;
        __syncwarp();
        const long long nck = status ? 0 : (total + K - 1) / K;
        for (long long c = nck - 1; c >= 0; --c) {
            const long long s0 = c * K, s1 = (s0 + K < total) ? s0 + K : total;
            for (int k = lane; k < np; k += 32) {
                nb[k] = my_ck[c * np_max + k];
                n1b[k] = 0.0;
            }
            __syncwarp();
            StepRec1 r = my_ckr[c];
            out_idx = r.out_idx;
            for (long long q = 0; q < s1 - s0; ++q) {
                if (q > 0) prepare(r);
                step(r, true, q);
            }
            __syncwarp();
            for (long long q = s1 - s0 - 1; q >= 0; --q) {
                const StepRec1 rr = my_sr[q];
                if (rr.clipped) {
                    const double* row = sd + (size_t)rr.out_idx * 6;
                    for (int k = 0; k < 4; ++k) pc[k] += row[1 + k];
                    lC += row[5];
                }
                double lV0 = Kn.kappa * lC, lCprev = lC;
                pc[3] += -Kn.kappa * lC;
                // stage-2 adjoint: input n1 (recorded), lam_eff = (lam + pc.W)/2
                for (int k = lane; k < np; k += 32) nb[k] = my_sn1[q * np_max + k];
                __syncwarp();
                double P1, P0;
                adj_stage(nb, lam, pc, 0.5, leff, fc, N, R, d1, P1, P0);
                for (int i = lane; i < N; i += 32) {
                    const double jt = fc[3 * (i + 2)] + fc[3 * (i + 1) + 1] + fc[3 * i + 2];
                    const double l2 = leff[i + 2];
                    lamo[i + 2] = l2;
                    u[i + 2] = l2 + rr.dt * rr.G1b * jt;
                }
                __syncwarp();
                double ldt = rr.G1b * P1 + rr.Bb * P0 / d1;
                double lC1 = 0.0, ltn = lt;
                kin_adj(Kn, rr.C1, rr.t_new, rr.dt * P1, rr.dt * P0 / d1, &lC1, &ltn, lth);
                lCprev += lC1;
                lV0 += Kn.kappa * lC1;
                double pu[4] = {0.0, 0.0, 0.0, -Kn.kappa * lC1};
                // stage-1 adjoint: input n (recorded), lam_eff = u + pu.W
                for (int k = lane; k < np; k += 32) nb[k] = my_sn[q * np_max + k];
                __syncwarp();
                adj_stage(nb, u, pu, 1.0, leff, fc, N, R, d1, P1, P0);
                for (int i = lane; i < N; i += 32) {
                    const double jt = fc[3 * (i + 2)] + fc[3 * (i + 1) + 1] + fc[3 * i + 2];
                    lamo[i + 2] += leff[i + 2] + rr.dt * rr.G1a * jt;
                }
                __syncwarp();
                ldt += rr.G1a * P1 + rr.Ba * P0 / d1;
                double lG1 = rr.dt * P1;
                const double lB = rr.dt * P0 / d1;
                double ltp;
                if (!rr.clipped) {
                    ltp = ltn;
                    ldt += ltn;
                    const double Rr = rr.G1a / d1;
                    lG1 += -Kn.cfl / (Rr * Rr) * ldt / d1;
                } else {
                    ltp = -ldt;
                }
                kin_adj(Kn, rr.C, rr.t, lG1, lB, &lCprev, &ltp, lth);
                lC = lCprev;
                lt = ltp;
                pc[0] = pc[1] = pc[2] = 0.0;
                pc[3] = lV0;
                double* tmp = lam;
                lam = lamo;
                lamo = tmp;
            }
        }
        if (row0) {
            for (int k = 0; k < 4; ++k) pc[k] += sd[1 + k];
            lC += sd[5];
        }
        if (dn0_out) {
            for (int i = lane; i < N; i += 32) {
                const double x = (i + 0.5) * d1;
                dn0_out[off + i] = lam[i + 2] + (pc[0] + x * (pc[1] + x * (pc[2] + x * pc[3]))) * d1;
            }
        }
        if (lane == 0) {
            for (int k = 0; k < 6; ++k) dth_out[(size_t)id * 7 + k] = lth[k];
            dth_out[(size_t)id * 7 + 6] = lC;
            status_out[id] = status;
        }
        __syncwarp();
    }
}

}  // namespace pbe

using namespace pbe;

struct pbe_batch;   // defined in pbe_batch.cu
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
}  // namespace

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
    pbe_batch_internal_view(b, &inst_v, &order, &count, &state, &Cs, &ts, &np_max, &device, &stream_v);
    {
        // the batched adjoint differentiates the power-law form (checked on the host copies)
        std::vector<BatchInst> hi(count);
        if (cudaMemcpy(hi.data(), inst_v, sizeof(BatchInst) * count, cudaMemcpyDeviceToHost) != cudaSuccess)
            return bafail(PBE_ECUDA, "reading the batch descriptors failed");
        for (int i = 0; i < count; ++i)
            if (hi[i].K.growth_form != 0 || hi[i].K.solubility_form != 0)
                return bafail(PBE_EINVAL, "instance %d: the batched adjoint needs power-law kinetics", i);
    }
    cudaStream_t st = (cudaStream_t)stream_v;
    const BatchInst* inst = (const BatchInst*)inst_v;
    const int K = checkpoint_every;
    const int max_ckpt = (4096 + K - 1) / K;   // up to 4096 steps per instance
    const int npa = np_max;   // per-instance buffer length (same layout as the forward batch)
    pbe_status rc = PBE_OK;
    double *ck = nullptr, *sn = nullptr, *sn1 = nullptr, *seeds = nullptr, *dth = nullptr, *dn0 = nullptr, *tout = nullptr;
    StepRec1 *ckr = nullptr, *sr = nullptr;
    int *status = nullptr;
    unsigned int* queue = nullptr;
    std::vector<double> h_dth((size_t)count * 7);
    std::vector<int> h_status(count);
    int wpb = 4, occ = 0, sms = 0, maxsm = 0;
    size_t smem = 0;
    long long slots = 0;
    const void* fn = nullptr;
    BATRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    BATRY(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    if (count < 1) goto out;
    while (wpb > 1 && (size_t)wpb * 10 * npa * sizeof(double) > (size_t)maxsm) wpb /= 2;
    // few instances per SM: spread them so every SM's FP64 pipe works on some
    while (wpb > 1 && (count + wpb - 1) / wpb < 2 * sms) wpb /= 2;
    smem = (size_t)wpb * 10 * npa * sizeof(double);
    if (smem > (size_t)maxsm) { rc = bafail(PBE_EINVAL, "instances too large for the batched adjoint"); goto out; }
    fn = wpb == 4 ? (const void*)k_batch_vjp<4> : (wpb == 2 ? (const void*)k_batch_vjp<2> : (const void*)k_batch_vjp<1>);
    BATRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    BATRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, wpb * 32, smem));
    if (occ < 1) { rc = bafail(PBE_ECUDA, "batched adjoint kernel does not fit on an SM"); goto out; }
    {
        int blocks = occ * sms;
        const int need = (count + wpb - 1) / wpb;
        if (blocks > need) blocks = need;
        slots = (long long)blocks * wpb;
        BATRY(cudaMalloc(&ck, sizeof(double) * slots * max_ckpt * npa));
        BATRY(cudaMalloc(&ckr, sizeof(StepRec1) * slots * max_ckpt));
        BATRY(cudaMalloc(&sn, sizeof(double) * slots * K * npa));
        BATRY(cudaMalloc(&sn1, sizeof(double) * slots * K * npa));
        BATRY(cudaMalloc(&sr, sizeof(StepRec1) * slots * K));
        BATRY(cudaMalloc(&seeds, sizeof(double) * (size_t)count * n_out * 6));
        BATRY(cudaMalloc(&dth, sizeof(double) * (size_t)count * 7));
        BATRY(cudaMalloc(&status, sizeof(int) * count));
        BATRY(cudaMalloc(&queue, sizeof(unsigned int)));
        BATRY(cudaMalloc(&tout, sizeof(double) * n_out));
        BATRY(cudaMemcpyAsync(seeds, seeds_in, sizeof(double) * (size_t)count * n_out * 6,
                              seeds_mem == PBE_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        BATRY(cudaMemcpyAsync(tout, t_out, sizeof(double) * n_out, cudaMemcpyHostToDevice, st));
        BATRY(cudaMemsetAsync(queue, 0, sizeof(unsigned int), st));
        double* dn0_dev = (dL_dn0 && mem == PBE_MEM_DEVICE) ? dL_dn0 : nullptr;
        int npa_arg = npa;
        void* args[] = {&inst, &order, &count, &state, &Cs, &ts, &tout, &n_out, &seeds, (void*)&K, (void*)&max_ckpt,
                        &ck, &ckr, &sn, &sn1, &sr, &dth, &dn0_dev, &status, &queue, &npa_arg};
        BATRY(cudaLaunchKernel(fn, blocks, wpb * 32, args, smem, st));
        BATRY(cudaMemcpyAsync(h_dth.data(), dth, sizeof(double) * (size_t)count * 7, cudaMemcpyDeviceToHost, st));
        BATRY(cudaMemcpyAsync(h_status.data(), status, sizeof(int) * count, cudaMemcpyDeviceToHost, st));
        BATRY(cudaStreamSynchronize(st));
    }
    for (int i = 0; i < count; ++i) {
        for (int k = 0; k < 6; ++k) dL_dtheta[(size_t)i * 6 + k] = h_dth[(size_t)i * 7 + k];
        if (dL_dC0) dL_dC0[i] = h_dth[(size_t)i * 7 + 6];
    }
    for (int i = 0; i < count; ++i)
        if (h_status[i] != PBE_OK) { rc = bafail(h_status[i], "instance %d: status %d in the batched adjoint", i, h_status[i]); break; }
out:
    cudaStreamSynchronize(st);
    cudaFree(ck); cudaFree(ckr); cudaFree(sn); cudaFree(sn1); cudaFree(sr); cudaFree(seeds); cudaFree(dth);
    cudaFree(status); cudaFree(queue); cudaFree(tout); cudaFree(dn0);
    return rc;
}

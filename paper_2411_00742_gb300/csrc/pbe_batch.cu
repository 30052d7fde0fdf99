// Batched 1-D solves: thousands of independent instances (own grid size,
// kinetics, cooling profile and CFL-limited step count) in one persistent
// launch.  One warp owns one instance at a time: its distribution and stage
// buffer live in the warp's slice of shared memory for the whole solve, the
// limiter stencil's neighbours come from shared memory and warp shuffles,
// the moment reductions are warp butterflies and the scalar chain runs on
// the warp's own lanes, so an instance never synchronizes with anything
// but its own warp.  Warps pull instance ids from an atomic queue ordered by
// estimated cost (longest first).  The launch is captured in a CUDA graph
// and replayed; the warps-per-block setting is chosen by pbe_batch_autotune.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "pbe_internal.h"
#include "pbe_tiles.cuh"

void pbe_set_error_message(int code, const char* msg);  // pbe_api.cu

namespace pbe {

constexpr int kMaxBatchCells = 6144;   // largest instance accepted (shared-memory resident)

// buffer layout per instance (cell i at index i + 2, two zero ghosts below)
__host__ __device__ inline int batch_np(int N) { return 32 * ((N + 31) / 32 + 1) + 3; }

template <int STAGE>
__device__ __forceinline__ void warp_stage(const double* in, const double* old, double* out, int N, int rows,
                                           double c1, double src, double d1, bool moms, double (&m)[4])
{
    const int lane = threadIdx.x & 31;
    // face f lies between cells f-1 (upwind) and f: (n_{f-2}, n_{f-1}, n_f) = in[f], in[f+1], in[f+2]
    double hcur = face_value<true>(in[lane], in[lane + 1], in[lane + 2]);
    double x = (lane + 0.5) * d1;
    const double dx32 = 32.0 * d1;
    for (int r = 0; r < rows; ++r) {
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
            const double w = v * d1;
            if (moms) {
                const double t1 = x * w, t2 = x * t1;
                m[0] += w; m[1] += t1; m[2] += t2; m[3] += x * t2;
            } else {
                m[3] += x * x * x * w;
            }
        }
        hcur = hnext;
        x += dx32;
    }
}

__device__ __forceinline__ double warp_allsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int WPB>
__global__ void __launch_bounds__(WPB * 32) k_batch1d(const BatchInst* __restrict__ inst, const int* __restrict__ order,
                                                      int count, double* state, double* Cst, double* tst,
                                                      const double* t_out, int n_out, double* rows,
                                                      long long* steps_out, int* status_out, unsigned int* queue,
                                                      int np_max, long long max_steps)
{
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* nb = smem + (size_t)warp * 2 * np_max;
    double* n1b = nb + np_max;
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = (int)atomicAdd(queue, 1u);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= count) break;
        const int id = order[idx];
        const Kin K = inst[id].K;
        const Geom g = inst[id].g;
        const long long off = inst[id].offset;
        const int N = g.N1, R = inst[id].rows;
        const int np = batch_np(N);
        for (int k = lane; k < np; k += 32) {
            const int i = k - 2;
            nb[k] = (i >= 0 && i < N) ? state[off + i] : 0.0;
            n1b[k] = 0.0;
        }
        __syncwarp();
        // scalar state (identical in every lane)
        Scal s;
        s.C = Cst[id];
        s.t = tst[id];
        s.steps = 0; s.status = 0; s.done = 0; s.out_idx = 0; s.n_out = n_out; s.max_steps = max_steps;
        double m[4] = {0.0, 0.0, 0.0, 0.0};
        {
            double x = (lane + 0.5) * g.d1;
            for (int i = lane; i < N; i += 32, x += 32.0 * g.d1) {
                const double w = nb[i + 2] * g.d1, t1 = x * w, t2 = x * t1;
                m[0] += w; m[1] += t1; m[2] += t2; m[3] += x * t2;
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) m[k] = warp_allsum(m[k]);
        s.V0 = m[3];
        double* my_rows = rows + (size_t)id * n_out * 6;
        if (!isfinite(m[0]) || !isfinite(m[3]) || !isfinite(s.C)) {
            s.status = PBE_ENONFINITE;
            s.done = 1;
        } else {
            while (s.out_idx < n_out && t_out[s.out_idx] == s.t) {
                if (lane == 0) {
                    double* row = my_rows + (size_t)s.out_idx * 6;
                    row[0] = s.t; row[1] = m[0]; row[2] = m[1]; row[3] = m[2]; row[4] = m[3]; row[5] = s.C;
                }
                s.out_idx += 1;
            }
            if (s.out_idx >= n_out) s.done = 1;
        }
        if (!s.done) {
            double G1, G2, B, dt, t_new;
            kinetics_warp<false>(K, s.C, s.t, G1, G2, B);
            s.clipped = timestep_fast(K, g, G1, G2, s.t, t_out[s.out_idx], dt, t_new);
            s.G1a = G1; s.Ba = B; s.dt = dt; s.t_new = t_new;
            if (!isfinite(G1) || !isfinite(B) || !isfinite(dt)) { s.status = PBE_ENONFINITE; s.done = 1; }
        }
        while (!s.done) {
            // stage 1: n1 = n + dt L(n)
            for (int k = 0; k < 4; ++k) m[k] = 0.0;
            warp_stage<1>(nb, nb, n1b, N, R, s.G1a * s.dt * g.inv_d1, s.dt * s.Ba * g.inv_d1, g.d1, false, m);
            const double V1 = warp_allsum(m[3]);
            __syncwarp();
            const double C1 = s.C - K.kappa * (V1 - s.V0);
            {
                double G1, G2, B;
                kinetics_warp<false>(K, C1, s.t_new, G1, G2, B);
                s.G1b = G1; s.Bb = B;
                if (!isfinite(V1) || !isfinite(G1) || !isfinite(B)) { s.status = PBE_ENONFINITE; s.done = 1; break; }
            }
            // stage 2: n = n/2 + (n1 + dt L(n1))/2
            const bool moms = s.clipped;
            for (int k = 0; k < 4; ++k) m[k] = 0.0;
            warp_stage<2>(n1b, nb, nb, N, R, s.G1b * s.dt * g.inv_d1, s.dt * s.Bb * g.inv_d1, g.d1, moms, m);
            if (moms) {
#pragma unroll
                for (int k = 0; k < 4; ++k) m[k] = warp_allsum(m[k]);
            } else {
                m[3] = warp_allsum(m[3]);
            }
            __syncwarp();
            const double V2 = m[3];
            s.C = s.C - K.kappa * (V2 - s.V0);
            s.t = s.t_new;
            s.V0 = V2;
            s.steps += 1;
            if (!isfinite(V2) || !isfinite(s.C)) { s.status = PBE_ENONFINITE; s.done = 1; break; }
            if (moms) {
                if (lane == 0) {
                    double* row = my_rows + (size_t)s.out_idx * 6;
                    row[0] = s.t; row[1] = m[0]; row[2] = m[1]; row[3] = m[2]; row[4] = m[3]; row[5] = s.C;
                }
                s.out_idx += 1;
            }
            if (s.out_idx >= n_out) { s.done = 1; break; }
            if (s.steps >= max_steps) { s.status = PBE_ETIMEOUT; s.done = 1; break; }
            double G1, G2, B, dt, t_new;
            kinetics_warp<false>(K, s.C, s.t, G1, G2, B);
            s.clipped = timestep_fast(K, g, G1, G2, s.t, t_out[s.out_idx], dt, t_new);
            s.G1a = G1; s.Ba = B; s.dt = dt; s.t_new = t_new;
            if (!isfinite(G1) || !isfinite(B) || !isfinite(dt)) { s.status = PBE_ENONFINITE; s.done = 1; }
        }
        __syncwarp();
        for (int i = lane; i < N; i += 32) state[off + i] = nb[i + 2];
        if (lane == 0) {
            Cst[id] = s.C;
            tst[id] = s.t;
            steps_out[id] = s.steps;
            status_out[id] = s.status;
        }
        __syncwarp();
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
    int wpb;                          // warps (instances) per block
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
    int exec_wpb, exec_nout;
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

const void* batch_kernel(int wpb)
{
    switch (wpb) {
        case 1: return (const void*)k_batch1d<1>;
        case 2: return (const void*)k_batch1d<2>;
        case 3: return (const void*)k_batch1d<3>;
        case 4: return (const void*)k_batch1d<4>;
        case 6: return (const void*)k_batch1d<6>;
        case 8: return (const void*)k_batch1d<8>;
        default: return nullptr;
    }
}

size_t batch_smem(const pbe_batch* b, int wpb) { return (size_t)wpb * 2 * b->np_max * sizeof(double); }

cudaError_t launch_batch(pbe_batch* b, int wpb, int n_out, cudaStream_t st)
{
    const void* fn = batch_kernel(wpb);
    size_t smem = batch_smem(b, wpb);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, wpb * 32, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) return e;
    int blocks = occ * sms;
    const int need = (b->count + wpb - 1) / wpb;
    if (blocks > need) blocks = need;
    e = cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    void* args[] = {&b->d_inst, &b->d_order, &b->count, &b->d_state, &b->d_C, &b->d_t, &b->d_tout, &n_out,
                    &b->d_rows, &b->d_steps, &b->d_status, &b->d_queue, &b->np_max, &b->max_steps};
    return cudaLaunchKernel(fn, blocks, wpb * 32, args, smem, st);
}

bool wpb_fits(const pbe_batch* b, int wpb)
{
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
    return batch_smem(b, wpb) <= (size_t)maxsm;
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
    if (!b->exec || b->exec_wpb != b->wpb || b->exec_nout != n_out) {
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        cudaStream_t cap;
        BTRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
        cudaError_t le = cudaSuccess;
        if (e == cudaSuccess) {
            le = launch_batch(b, b->wpb, n_out, cap);
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
    for (int i = 0; i < count; ++i) {
        const pbe_instance& p = inst[i];
        const pbe_kinetics* k = &p.kin;
        if (p.ncells < 1 || p.ncells > kMaxBatchCells) {
            delete b;
            return bfail(PBE_EINVAL, "instance %d: ncells = %lld outside [1, %d]", i, (long long)p.ncells, kMaxBatchCells);
        }
        if (!(p.lmax > 0.0) || !std::isfinite(p.lmax) || !std::isfinite(p.C0) || !std::isfinite(p.t0) ||
            !(k->cfl > 0.0 && k->cfl <= 1.0) || !(k->t_cool > 0.0) ||
            (k->kind != PBE_KINETICS_POWER_LAW && k->kind != PBE_KINETICS_FIXED) || k->kg[0] < 0 || k->kb < 0 ||
            k->scheme != PBE_SCHEME_SSPRK2 || (k->growth_form != 0 && k->growth_form != 1) ||
            (k->solubility_form != 0 && k->solubility_form != 1)) {
            // (the learned closure runs on the single-grid plain path only)
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
    b->np_max = batch_np(nmax);
    b->wpb = 4;
    b->max_steps = 1000000;
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return bfail(PBE_ECUDA, "no CUDA device available");
    }
    bool ok = cudaMalloc(&b->d_inst, sizeof(BatchInst) * count) == cudaSuccess &&
              cudaMalloc(&b->d_order, sizeof(int) * count) == cudaSuccess &&
              cudaMalloc(&b->d_state, sizeof(double) * b->total_cells) == cudaSuccess &&
              cudaMalloc(&b->d_C, sizeof(double) * count) == cudaSuccess &&
              cudaMalloc(&b->d_t, sizeof(double) * count) == cudaSuccess &&
              cudaMalloc(&b->d_steps, sizeof(long long) * count) == cudaSuccess &&
              cudaMalloc(&b->d_status, sizeof(int) * count) == cudaSuccess &&
              cudaMalloc(&b->d_queue, sizeof(unsigned int)) == cudaSuccess &&
              cudaMallocHost(&b->h_steps, sizeof(long long) * count) == cudaSuccess &&
              cudaMallocHost(&b->h_status, sizeof(int) * count) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        pbe_batch_destroy(b);
        return bfail(PBE_ENOMEM, "allocating the batch failed");
    }
    if (cudaMemcpy(b->d_inst, h.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
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

pbe_status pbe_batch_steps(pbe_batch* b, int64_t* steps)
{
    if (!b || !steps) return bfail(PBE_EINVAL, "null argument");
    for (int i = 0; i < b->count; ++i) steps[i] = b->h_steps[i];
    return PBE_OK;
}

pbe_status pbe_batch_set_config(pbe_batch* b, int warps_per_block)
{
    if (!b) return bfail(PBE_EINVAL, "null batch");
    if (!batch_kernel(warps_per_block)) return bfail(PBE_EINVAL, "warps_per_block must be 1, 2, 3, 4, 6 or 8");
    if (!wpb_fits(b, warps_per_block))
        return bfail(PBE_EINVAL, "%d instances of up to %d cells do not fit in one block's shared memory",
                     warps_per_block, (b->np_max - 35));
    b->wpb = warps_per_block;
    return PBE_OK;
}

pbe_status pbe_batch_solve(pbe_batch* b, const double* t_out, int n_out, double* rows, int mem, int64_t* total_steps)
{
    if (!b || !rows) return bfail(PBE_EINVAL, "null argument");
    pbe_status st = check_times(b, t_out, n_out);
    if (st) return st;
    for (int i = 0; i < b->count; ++i)
        if (t_out[0] < b->t0[i]) return bfail(PBE_EINVAL, "t_out[0] precedes instance %d's start time", i);
    if (!wpb_fits(b, b->wpb)) {
        int w = b->wpb;
        while (w > 1 && !wpb_fits(b, w)) w /= 2;
        b->wpb = w;
    }
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
    BTRY(cudaMemcpyAsync(save, b->d_state, sizeof(double) * b->total_cells, cudaMemcpyDeviceToDevice, b->stream));
    BTRY(cudaMemcpyAsync(saveC, b->d_C, sizeof(double) * b->count, cudaMemcpyDeviceToDevice, b->stream));
    BTRY(cudaMemcpyAsync(savet, b->d_t, sizeof(double) * b->count, cudaMemcpyDeviceToDevice, b->stream));
    BTRY(cudaMemcpyAsync(b->d_tout, t_out, sizeof(double) * n_out, cudaMemcpyHostToDevice, b->stream));
    cudaEvent_t e0, e1;
    BTRY(cudaEventCreate(&e0));
    BTRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_w = b->wpb;
    const int cands[] = {1, 2, 3, 4, 6, 8};
    for (int w : cands) {
        if (!wpb_fits(b, w)) continue;
        float tsum = 0.0f;
        for (int rep = 0; rep < 2; ++rep) {
            BTRY(cudaMemcpyAsync(b->d_state, save, sizeof(double) * b->total_cells, cudaMemcpyDeviceToDevice, b->stream));
            BTRY(cudaMemcpyAsync(b->d_C, saveC, sizeof(double) * b->count, cudaMemcpyDeviceToDevice, b->stream));
            BTRY(cudaMemcpyAsync(b->d_t, savet, sizeof(double) * b->count, cudaMemcpyDeviceToDevice, b->stream));
            BTRY(cudaEventRecord(e0, b->stream));
            BTRY(launch_batch(b, w, n_out, b->stream));
            BTRY(cudaEventRecord(e1, b->stream));
            BTRY(cudaEventSynchronize(e1));
            float ms;
            BTRY(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) tsum += ms;   // first run warms up
        }
        if (tsum < best) { best = tsum; best_w = w; }
    }
    BTRY(cudaMemcpyAsync(b->d_state, save, sizeof(double) * b->total_cells, cudaMemcpyDeviceToDevice, b->stream));
    BTRY(cudaMemcpyAsync(b->d_C, saveC, sizeof(double) * b->count, cudaMemcpyDeviceToDevice, b->stream));
    BTRY(cudaMemcpyAsync(b->d_t, savet, sizeof(double) * b->count, cudaMemcpyDeviceToDevice, b->stream));
    BTRY(cudaStreamSynchronize(b->stream));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(save); cudaFree(saveC); cudaFree(savet);
    b->wpb = best_w;
    if (chosen) *chosen = best_w;
    return PBE_OK;
}

}  // extern "C"

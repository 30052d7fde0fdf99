// pbe_solve_1d_noalloc: a 1-D solve that allocates no memory at all.
//
// Who needs this: callers that must not allocate device or host memory once
// they are running - for example code that runs inside a real-time control
// loop with a fixed memory budget, code embedded in another framework's
// allocator-managed process that forbids foreign cudaMalloc calls, or a
// caller that already holds every byte of device memory it may use.  The
// grid-based API (pbe_create_grid) allocates its state and work buffers;
// this entry point takes the caller's buffers for inputs and outputs and
// keeps its own working memory in one fixed array that is part of the
// library image.
//
// Working memory: g_noalloc_scratch below, a file-scope __device__ array of
// kScratchDoubles doubles (about 0.56 MB).  Every GPU that loads this library
// carries it until the process exits.  All calls share it, and it keeps the
// contents of the last call; the scalar header is cleared before each solve.
// Two calls whose work overlaps on a GPU (different streams, or different
// host threads) race on it and give wrong results: serialize them.
#include <cstring>
#include <mutex>
#include <string>

#include "pbe_internal.h"
#include "pbe_tiles.cuh"

void pbe_set_error_message(int code, const char* msg);  // defined in pbe_api.cu

namespace {

constexpr int kNT = 256;
constexpr int kTile = 1024;
constexpr int64_t kMaxCells = 1 << 16;     // largest grid accepted
constexpr int kMaxOut = 4096;              // largest number of output times accepted
constexpr int kHeaderDoubles = 64;         // scalar block (pbe::Scal) at the start
constexpr int64_t kScratchDoubles = kHeaderDoubles + kMaxOut + kMaxCells;
static_assert(sizeof(pbe::Scal) <= kHeaderDoubles * sizeof(double), "scalar header too small");

// Host code must not take the address of this array directly: in host code
// the name is only a stand-in, so its device address is looked up with
// cudaGetSymbolAddress once per device (see scratch_ptr).
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

using namespace pbe;

// Whole solve in one block: the block walks the tiles of each stage in turn,
// so the stage boundaries need only __syncthreads, and the scalar chain is
// kept in shared memory.  Same arithmetic as the plain path's stage kernels.
__global__ void __launch_bounds__(kNT) k_solve1d_noalloc(double* n, double* scratch, Kin K, Geom g, int n_out,
                                                         double* rows, long long max_steps)
{
    Scal* S = reinterpret_cast<Scal*>(scratch);
    const double* t_out = scratch + kHeaderDoubles;
    double* n1 = scratch + kHeaderDoubles + kMaxOut;
    __shared__ double tile[kTile + 3];
    __shared__ double h[kTile + 1];
    __shared__ double sh[kNT / 32 * 4];
    __shared__ Scal s;
    const int N = g.N1;
    const int ntiles = (N + kTile - 1) / kTile;

    // prologue: moments of n, rows at the current time, first step
    double m[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < N; i += kNT) {
        double x = (i + 0.5) * g.d1, v = n[i] * g.d1;
        m[0] += v; m[1] += x * v; m[2] += x * x * v; m[3] += x * x * x * v;
    }
    block_sum<kNT, 4>(m, sh);
    if (threadIdx.x == 0) {
        s = *S;  // C and t were written by the host into the cleared header
        s.V0 = m[3];
        s.steps = 0; s.status = 0; s.done = 0; s.out_idx = 0; s.n_out = n_out; s.max_steps = max_steps;
        s.counter = 0u;
        if (!isfinite(m[0]) || !isfinite(m[3]) || !isfinite(s.C)) {
            s.status = PBE_ENONFINITE;
            s.done = 1;
        } else {
            while (s.out_idx < n_out && t_out[s.out_idx] == s.t) {
                double* row = rows + (size_t)s.out_idx * 6;
                row[0] = s.t;
                for (int k = 0; k < 4; ++k) row[1 + k] = m[k];
                row[5] = s.C;
                s.out_idx += 1;
            }
            if (s.out_idx >= n_out) s.done = 1;
            else prepare_step(&s, K, g, t_out);
        }
    }
    __syncthreads();
    while (!s.done) {
        StageCoef sc = stage_coef<1>(s, g);
        for (int k = 0; k < 4; ++k) m[k] = 0.0;
        for (int t = 0; t < ntiles; ++t) tile1d<1, true, false, kTile, kNT>(n, n, n1, t * kTile, g, sc, m, tile, h);
        block_sum<kNT, 4>(m, sh);
        if (threadIdx.x == 0) finish_stage1(&s, K, m[3]);
        __syncthreads();
        if (s.done) break;
        sc = stage_coef<2>(s, g);
        for (int k = 0; k < 4; ++k) m[k] = 0.0;
        for (int t = 0; t < ntiles; ++t) tile1d<2, true, false, kTile, kNT>(n1, n, n, t * kTile, g, sc, m, tile, h);
        block_sum<kNT, 4>(m, sh);
        if (threadIdx.x == 0) finish_stage2(&s, K, g, t_out, rows, m, 4, 3);
        __syncthreads();
    }
    if (threadIdx.x == 0) *S = s;
}

// Device address of the scratch array, looked up once per device with that
// device current.
double* scratch_ptr(int dev, cudaError_t* err)
{
    static std::mutex mu;
    static double* ptrs[64] = {nullptr};
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    if (!ptrs[dev]) {
        void* p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (*err != cudaSuccess) return nullptr;
        ptrs[dev] = static_cast<double*>(p);
    }
    *err = cudaSuccess;
    return ptrs[dev];
}

pbe_status fail(int code, const std::string& msg)
{
    pbe_set_error_message(code, msg.c_str());
    return code;
}

}  // namespace

extern "C" pbe_status pbe_solve_1d_noalloc(const pbe_kinetics* k, int64_t ncells, double lmax, double* n,
                                           double C0, double t0, const double* t_out, int n_out, double* rows,
                                           int64_t* steps, void* stream)
{
    if (!k || !n || !t_out || !rows) return fail(PBE_EINVAL, "null argument");
    if (ncells < 1 || ncells > kMaxCells)
        return fail(PBE_EINVAL, "ncells = " + std::to_string((long long)ncells) +
                                    " outside [1, 65536], the limit of the fixed scratch array");
    if (n_out < 1 || n_out > kMaxOut)
        return fail(PBE_EINVAL, "n_out = " + std::to_string(n_out) + " outside [1, 4096], the limit of the fixed scratch array");
    if (!(lmax > 0.0) || !std::isfinite(lmax)) return fail(PBE_EINVAL, "lmax must be positive and finite");
    if (!std::isfinite(C0) || !std::isfinite(t0)) return fail(PBE_EINVAL, "non-finite C0 or t0");
    if (k->kind != PBE_KINETICS_POWER_LAW && k->kind != PBE_KINETICS_FIXED) return fail(PBE_EINVAL, "unknown kinetics kind");
    if (k->scheme != PBE_SCHEME_SSPRK2 || k->growth_form != 0 || k->solubility_form != 0)
        return fail(PBE_EINVAL, "this entry point runs the SSP-RK2 scheme with power-law kinetics");
    if (check_kinetic_values(k) != PBE_OK) return PBE_EINVAL;   // message set by the check
    if (!(t_out[0] >= t0) || !std::isfinite(t_out[0])) return fail(PBE_EINVAL, "t_out[0] precedes t0");
    for (int j = 1; j < n_out; ++j)
        if (!(t_out[j] > t_out[j - 1]) || !std::isfinite(t_out[j]))
            return fail(PBE_EINVAL, "t_out must be strictly increasing and finite");
    int dev;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PBE_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    double* scratch = scratch_ptr(dev, &e);
    if (!scratch) return fail(PBE_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;

    Kin K;
    memset(&K, 0, sizeof(K));
    K.kind = k->kind; K.ndim = 1;
    K.kg1 = k->kg[0]; K.g1 = k->g[0]; K.kg2 = 0.0; K.g2 = 1.0; K.kb = k->kb; K.b = k->b;
    K.cs0 = k->csat[0]; K.cs1 = k->csat[1]; K.cs2 = k->csat[2];
    K.T0 = k->T0; K.T1 = k->T1; K.t_cool = k->t_cool; K.kappa = k->kappa; K.cfl = k->cfl;
    K.lkg1 = std::log(K.kg1); K.lkg2 = 0.0; K.lkb = std::log(K.kb);
    K.inv_tcool = 1.0 / K.t_cool;
    Geom g;
    g.ndim = 1; g.N1 = (int)ncells; g.N2 = 1; g.d1 = lmax / (double)ncells; g.d2 = 1.0;
    g.inv_d1 = 1.0 / g.d1; g.inv_d2 = 1.0;

    // clear the scalar header, then place C0 and t0 and the output times in the scratch
    Scal hs;
    memset(&hs, 0, sizeof(hs));
    hs.C = C0;
    hs.t = t0;
    if ((e = cudaMemcpyAsync(scratch, &hs, sizeof(hs), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(scratch + kHeaderDoubles, t_out, sizeof(double) * n_out, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
        return fail(PBE_ECUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    k_solve1d_noalloc<<<1, kNT, 0, st>>>(n, scratch, K, g, n_out, rows, 1000000LL);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(PBE_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    // read the scalar header back (status and step count) into host stack memory
    if ((e = cudaMemcpyAsync(&hs, scratch, sizeof(hs), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(PBE_ECUDA, std::string("readback: ") + cudaGetErrorString(e));
    if (steps) *steps = hs.steps;
    if (hs.status == PBE_ENONFINITE) return fail(PBE_ENONFINITE, "non-finite value in the state or kinetics");
    if (hs.status == PBE_ETIMEOUT) return fail(PBE_ETIMEOUT, "step budget of 1e6 steps exhausted");
    if (hs.status != PBE_OK) return fail(hs.status, "device reported an error");
    return PBE_OK;
}

// C ABI of the solver (include/pbe.h): argument checking, device buffers,
// stream ordering and the solve loop.  All arithmetic runs in the kernels of
// pbe_plain.cu / pbe_fused.cu.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "pbe_internal.h"

using pbe::Scal;

static thread_local char g_err[512] = "";

static pbe_status fail(pbe_status code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

// Lets other translation units of the library report an error through
// pbe_last_error().
void pbe_set_error_message(int code, const char* msg)
{
    (void)code;
    snprintf(g_err, sizeof(g_err), "%s", msg);
}

#define CUDA_TRY(call)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(PBE_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                        __FILE__, __LINE__);                                                 \
    } while (0)

namespace {
// Makes the grid's device current for the duration of a call and restores
// the caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

cudaMemcpyKind kind_to_device(int mem) { return mem == PBE_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
cudaMemcpyKind kind_from_device(int mem) { return mem == PBE_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

void free_grid_buffers(pbe_grid* g)
{
    pbe::adjoint_work_free(g);
    if (g->plain_exec) cudaGraphExecDestroy(g->plain_exec);
    cudaFree(g->d_n); cudaFree(g->d_n1); cudaFree(g->d_S); cudaFree(g->d_part); cudaFree(g->d_mom); cudaFree(g->d_bar);
    cudaFree(g->d_tout); cudaFree(g->d_rows); cudaFree(g->d_rowpart); cudaFree(g->d_poly);
    cudaFreeHost(g->h_S); cudaFreeHost(g->h_stage); cudaFreeHost(g->h_tout);
    if (g->ev_k0) cudaEventDestroy(g->ev_k0);
    if (g->ev_k1) cudaEventDestroy(g->ev_k1);
}

int ncol_of(const pbe_grid* g) { return g->geo.ndim == 1 ? 6 : 12; }

pbe_status ensure_tout_capacity(pbe_grid* g, int n_out)
{
    if (n_out <= g->tout_cap) return PBE_OK;
    int cap = g->tout_cap ? g->tout_cap : 64;
    while (cap < n_out) cap *= 2;
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    cudaFree(g->d_tout); cudaFree(g->d_rows); cudaFree(g->d_rowpart); cudaFreeHost(g->h_tout);
    g->d_tout = nullptr; g->d_rows = nullptr; g->d_rowpart = nullptr; g->h_tout = nullptr; g->tout_cap = 0;
    g->tout_valid_n = 0;
    if (g->plain_exec) { cudaGraphExecDestroy(g->plain_exec); g->plain_exec = nullptr; }
    if (cudaMalloc(&g->d_tout, sizeof(double) * cap) != cudaSuccess ||
        cudaMalloc(&g->d_rows, sizeof(double) * cap * 12) != cudaSuccess ||
        cudaMalloc(&g->d_rowpart, sizeof(double) * (size_t)cap * (g->max_blocks / 2 + 1) * 10) != cudaSuccess ||
        cudaMallocHost(&g->h_tout, sizeof(double) * cap) != cudaSuccess)
        return fail(PBE_ENOMEM, "cudaMalloc of %d output rows failed", cap);
    g->tout_cap = cap;
    return PBE_OK;
}

// Graph of the plain loop: a conditional while node whose body is the two
// stage kernels; the last block of stage 2 clears the condition when the
// solve is done (all output times reached, an error, or the step budget).
pbe_status build_plain_graph(pbe_grid* g)
{
    if (g->plain_exec || g->plain_graph_failed) return PBE_OK;
    cudaGraph_t graph = nullptr;
    cudaStream_t cap = nullptr;
    cudaStream_t saved = g->stream;
    cudaGraphConditionalHandle h;
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cudaGraphNode_t node;
    cudaGraph_t body, captured;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    }
    if (e == cudaSuccess) {
        body = cp.conditional.phGraph_out[0];
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    }
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        g->stream = cap;
        cudaError_t le = pbe::launch_plain_step(g, true, h);
        g->stream = saved;
        e = cudaStreamEndCapture(cap, &captured);
        if (e == cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->plain_exec, graph, 0);
    if (cap) cudaStreamDestroy(cap);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g->plain_exec = nullptr;
        g->plain_graph_failed = true;  // the host loop below stays available
        cudaGetLastError();
    }
    return PBE_OK;
}

pbe_status finish_call(pbe_grid* g)
{
    CUDA_TRY(cudaMemcpyAsync(g->h_S, g->d_S, sizeof(Scal), cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    g->C_host = g->h_S->C;
    g->t_host = g->h_S->t;
    int st = g->h_S->status;
    if (st == PBE_ENONFINITE) return fail(st, "non-finite value in the state or kinetics at t = %g", g->h_S->t);
    if (st == PBE_ETIMEOUT) return fail(st, "step budget of %lld steps exhausted at t = %g", g->h_S->max_steps, g->h_S->t);
    if (st != PBE_OK) return fail(st, "device reported status %d", st);
    return PBE_OK;
}

pbe_status run_solve(pbe_grid* g, int n_out)
{
    CUDA_TRY(pbe::launch_prologue(g, n_out, g->max_steps, nullptr));
    if (g->path == PBE_PATH_FUSED && pbe::fused_supported(g) && g->kin.scheme == PBE_SCHEME_SSPRK2) {
        // the closure and the polynomial growth law: the persistent kernel's forward pass
        if (g->kin.kind == PBE_KINETICS_MLP || g->kin.growth_form == 2) CUDA_TRY(pbe::launch_solve_persistent(g, n_out));
        else CUDA_TRY(pbe::launch_fused_solve(g, n_out));
        return PBE_OK;
    }
    build_plain_graph(g);
    if (g->plain_exec) {
        if (g->timing) CUDA_TRY(cudaEventRecord(g->ev_k0, g->stream));
        CUDA_TRY(cudaGraphLaunch(g->plain_exec, g->stream));
        if (g->timing) CUDA_TRY(cudaEventRecord(g->ev_k1, g->stream));
        CUDA_TRY(pbe::launch_paper_finish(g));
        return PBE_OK;
    }
    // host loop over chunks of steps; stage kernels return at once when done
    if (g->timing) CUDA_TRY(cudaEventRecord(g->ev_k0, g->stream));
    for (long long done_steps = 0;;) {
        int chunk = 16;
        for (int k = 0; k < chunk; ++k) CUDA_TRY(pbe::launch_plain_step(g, false, 0));
        done_steps += chunk;
        CUDA_TRY(cudaMemcpyAsync(g->h_S, g->d_S, sizeof(Scal), cudaMemcpyDeviceToHost, g->stream));
        CUDA_TRY(cudaStreamSynchronize(g->stream));
        if (g->h_S->done) break;
        if (done_steps > g->max_steps + chunk) return fail(PBE_ETIMEOUT, "solve did not finish");
    }
    if (g->timing) CUDA_TRY(cudaEventRecord(g->ev_k1, g->stream));
    CUDA_TRY(pbe::launch_paper_finish(g));
    return PBE_OK;
}
}  // namespace

pbe_status pbe::prepare_tout(pbe_grid* g, const double* t_out, int n_out)
{
    pbe_status st = ensure_tout_capacity(g, n_out);
    if (st) return st;
    // the output times go to the device only when they changed since the last solve
    if (n_out != g->tout_valid_n || memcmp(g->h_tout, t_out, sizeof(double) * n_out) != 0) {
        memcpy(g->h_tout, t_out, sizeof(double) * n_out);
        CUDA_TRY(cudaMemcpyAsync(g->d_tout, g->h_tout, sizeof(double) * n_out, cudaMemcpyHostToDevice, g->stream));
        g->tout_valid_n = n_out;
    }
    return PBE_OK;
}

// The value checks every entry point applies to a pbe_kinetics: every
// parameter finite, rate prefactors not negative (a negative growth rate
// would reverse the upwind direction the stencil assumes), cfl in (0, 1],
// t_cool > 0.  Sets the thread's error message on failure.
pbe_status pbe::check_kinetic_values(const pbe_kinetics* k)
{
    const double vals[] = {k->kg[0], k->kg[1], k->g[0], k->g[1], k->kb, k->b, k->csat[0], k->csat[1],
                           k->csat[2], k->T0, k->T1, k->t_cool, k->kappa, k->cfl, k->ea[0], k->ea[1]};
    for (double v : vals)
        if (!std::isfinite(v)) return fail(PBE_EINVAL, "non-finite kinetic parameter");
    if (k->kg[0] < 0 || k->kg[1] < 0 || k->kb < 0) return fail(PBE_EINVAL, "negative rate prefactor");
    if (!(k->cfl > 0.0 && k->cfl <= 1.0)) return fail(PBE_EINVAL, "cfl must lie in (0, 1]");
    if (!(k->t_cool > 0.0)) return fail(PBE_EINVAL, "t_cool must be positive");
    return PBE_OK;
}

namespace pbe {
// The flat closure layout W1, b1, W2, b2, W3, b3 split into the bf16
// matrices and fp32 biases the kernels read.
void pack_closure(const float* w, std::vector<__nv_bfloat16>& hw, std::vector<float>& hb)
{
    const int H = kMlpH;
    hw.assign(H * 3 + H * H + 3 * H, __float2bfloat16_rn(0.0f));
    hb.assign(H + H + 3, 0.0f);
    const float* W1 = w;
    const float* b1 = W1 + H * 3;
    const float* W2 = b1 + H;
    const float* b2 = W2 + H * H;
    const float* W3 = b2 + H;
    const float* b3 = W3 + 3 * H;
    for (int k = 0; k < H * 3; ++k) hw[k] = __float2bfloat16_rn(W1[k]);
    for (int k = 0; k < H * H; ++k) hw[H * 3 + k] = __float2bfloat16_rn(W2[k]);
    for (int k = 0; k < 3 * H; ++k) hw[H * 3 + H * H + k] = __float2bfloat16_rn(W3[k]);
    for (int k = 0; k < H; ++k) { hb[k] = b1[k]; hb[H + k] = b2[k]; }
    for (int k = 0; k < 3; ++k) hb[2 * H + k] = b3[k];
}
}  // namespace pbe

extern "C" {

const char* pbe_last_error(void) { return g_err; }

int pbe_version(void) { return 100; }

pbe_status pbe_create_grid(pbe_grid** out, int ndim, const int64_t* ncells, const double* lmax)
{
    if (!out || !ncells || !lmax) return fail(PBE_EINVAL, "null argument");
    *out = nullptr;
    if (ndim != 1 && ndim != 2) return fail(PBE_EINVAL, "ndim must be 1 or 2 (got %d)", ndim);
    for (int d = 0; d < ndim; ++d) {
        if (ncells[d] < 1 || ncells[d] > (1LL << 20))
            return fail(PBE_EINVAL, "ncells[%d] = %lld out of range [1, 2^20]", d, (long long)ncells[d]);
        if (!(lmax[d] > 0.0) || !std::isfinite(lmax[d]))
            return fail(PBE_EINVAL, "lmax[%d] must be positive and finite", d);
    }
    long long nc = ncells[0] * (ndim == 2 ? ncells[1] : 1);
    if (nc > (1LL << 31)) return fail(PBE_EINVAL, "grid of %lld cells is too large", nc);
    pbe_grid* g = new pbe_grid();
    memset((void*)g, 0, sizeof(*g));
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        delete g;
        return fail(PBE_ECUDA, "no CUDA device available");
    }
    g->geo.ndim = ndim;
    g->geo.N1 = (int)ncells[0];
    g->geo.N2 = ndim == 2 ? (int)ncells[1] : 1;
    g->geo.d1 = lmax[0] / (double)ncells[0];
    g->geo.d2 = ndim == 2 ? lmax[1] / (double)ncells[1] : 1.0;
    g->geo.inv_d1 = 1.0 / g->geo.d1;
    g->geo.inv_d2 = 1.0 / g->geo.d2;
    g->ncell = (size_t)nc;
    g->path = PBE_PATH_PLAIN;
    g->max_steps = 1000000;
    g->wait_cycles = -1;
    g->kernel_ms = -1.0;
    if (cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess || g->sms < 1)
        g->sms = 1;
    g->window_mode = -1;
    if (ndim == 2 && pbe::window_setup() != cudaSuccess) {
        delete g;
        return fail(PBE_ECUDA, "cannot configure the 2-D stage kernels");
    }
    g->max_blocks = pbe::plain_max_blocks(g->geo);
    if (g->max_blocks < 1024) g->max_blocks = 1024;
    bool ok = cudaMalloc(&g->d_n, sizeof(double) * nc) == cudaSuccess &&
              cudaMalloc(&g->d_n1, sizeof(double) * nc) == cudaSuccess &&
              cudaMalloc(&g->d_S, sizeof(Scal)) == cudaSuccess &&
              cudaMalloc(&g->d_part, sizeof(double) * pbe::kMaxMom * g->max_blocks) == cudaSuccess &&
              cudaMalloc(&g->d_mom, sizeof(double) * pbe::kMaxMom) == cudaSuccess &&
              cudaMalloc(&g->d_bar, 512) == cudaSuccess &&
              cudaMallocHost(&g->h_S, sizeof(Scal)) == cudaSuccess &&
              cudaMallocHost(&g->h_stage, sizeof(double) * 64) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_grid_buffers(g);
        delete g;
        return fail(PBE_ENOMEM, "allocation of grid buffers failed");
    }
    // per-thread default stream: no device-wide synchronization, so grids can
    // be created while other threads' solves and graph captures are in flight
    if (cudaMemsetAsync(g->d_S, 0, sizeof(Scal), cudaStreamPerThread) != cudaSuccess ||
        cudaMemsetAsync(g->d_n, 0, sizeof(double) * nc, cudaStreamPerThread) != cudaSuccess ||
        cudaStreamSynchronize(cudaStreamPerThread) != cudaSuccess) {
        free_grid_buffers(g);
        delete g;
        return fail(PBE_ECUDA, "initialising grid buffers failed");
    }
    *out = g;
    return PBE_OK;
}

pbe_status pbe_destroy_grid(pbe_grid* g)
{
    if (!g) return PBE_OK;
    DeviceGuard dg(g->device);
    cudaStreamSynchronize(g->stream);
    free_grid_buffers(g);
    delete g;
    return PBE_OK;
}

pbe_status pbe_set_stream(pbe_grid* g, void* stream)
{
    if (!g) return fail(PBE_EINVAL, "null grid");
    g->stream = (cudaStream_t)stream;
    return PBE_OK;
}

pbe_status pbe_set_path(pbe_grid* g, int path)
{
    if (!g) return fail(PBE_EINVAL, "null grid");
    if (path != PBE_PATH_PLAIN && path != PBE_PATH_FUSED && path != PBE_PATH_AUTO)
        return fail(PBE_EINVAL, "unknown path %d", path);
    g->path = path == PBE_PATH_AUTO ? PBE_PATH_FUSED : path;   // fused falls back to plain where it does not apply
    return PBE_OK;
}

pbe_status pbe_set_window(pbe_grid* g, int mode)
{
    if (!g) return fail(PBE_EINVAL, "null grid");
    if (mode < -1 || mode > 1) return fail(PBE_EINVAL, "window mode must be -1, 0 or 1 (got %d)", mode);
    if (mode != g->window_mode && g->plain_exec) {   // the graph holds the previous kernels
        cudaGraphExecDestroy(g->plain_exec);
        g->plain_exec = nullptr;
    }
    if (mode != g->window_mode) g->fused_fn = nullptr;   // the fused launch shape is chosen again
    g->window_mode = mode;
    return PBE_OK;
}

pbe_status pbe_set_block_limit(pbe_grid* g, int blocks)
{
    if (!g) return fail(PBE_EINVAL, "null grid");
    if (blocks < 0) return fail(PBE_EINVAL, "block limit must be >= 0 (got %d)", blocks);
    if (blocks != g->block_limit) {
        // the launch shapes are chosen again (the adjoint's buffers with them)
        CUDA_TRY(cudaStreamSynchronize(g->stream));
        g->fused_fn = nullptr;
        pbe::adjoint_work_free(g);
        g->block_limit = blocks;
    }
    return PBE_OK;
}

pbe_status pbe_set_wait_limit(pbe_grid* g, double seconds)
{
    if (!g) return fail(PBE_EINVAL, "null grid");
    if (seconds < 0.0) {
        g->wait_cycles = -1;
        return PBE_OK;
    }
    int khz = 0;
    if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, g->device) != cudaSuccess || khz <= 0) khz = 2000000;
    g->wait_cycles = (long long)(seconds * 1e3 * (double)khz);
    return PBE_OK;
}

pbe_status pbe_set_max_steps(pbe_grid* g, int64_t max_steps)
{
    if (!g || max_steps < 1) return fail(PBE_EINVAL, "max_steps must be >= 1");
    g->max_steps = max_steps;
    return PBE_OK;
}

pbe_status pbe_set_kinetics(pbe_grid* g, const pbe_kinetics* k)
{
    if (!g || !k) return fail(PBE_EINVAL, "null argument");
    if (k->kind != PBE_KINETICS_POWER_LAW && k->kind != PBE_KINETICS_FIXED && k->kind != PBE_KINETICS_MLP)
        return fail(PBE_EINVAL, "unknown kinetics kind %d", k->kind);
    if (k->kind == PBE_KINETICS_MLP && !g->d_mW)
        return fail(PBE_ESTATE, "set the closure weights (pbe_set_closure) before selecting PBE_KINETICS_MLP");
    if (!(k->cfl > 0.0 && k->cfl <= 1.0)) return fail(PBE_EINVAL, "cfl must lie in (0, 1]");
    if (!(k->t_cool > 0.0)) return fail(PBE_EINVAL, "t_cool must be positive");
    if (k->scheme != PBE_SCHEME_SSPRK2 && k->scheme != PBE_SCHEME_PAPER) return fail(PBE_EINVAL, "unknown scheme %d", k->scheme);
    if ((k->growth_form < 0 || k->growth_form > 2) || (k->solubility_form != 0 && k->solubility_form != 1))
        return fail(PBE_EINVAL, "unknown growth or solubility form");
    if (k->scheme == PBE_SCHEME_PAPER && k->kind == PBE_KINETICS_MLP)
        return fail(PBE_EINVAL, "the learned closure runs with the SSP-RK2 scheme");
    if (k->growth_form == 2 && k->kind != PBE_KINETICS_POWER_LAW)
        return fail(PBE_EINVAL, "the polynomial growth law replaces the power law (kind PBE_KINETICS_POWER_LAW)");
    if (k->growth_form == 2 && !g->d_poly)
        return fail(PBE_ESTATE, "set the growth polynomial (pbe_set_growth_poly) before selecting growth_form 2");
    pbe_status pst = pbe::check_kinetic_values(k);
    if (pst != PBE_OK) return pst;
    pbe::Kin K;
    K.kind = k->kind;
    K.ndim = g->geo.ndim;
    K.kg1 = k->kg[0]; K.g1 = k->g[0]; K.kg2 = k->kg[1]; K.g2 = k->g[1]; K.kb = k->kb; K.b = k->b;
    K.cs0 = k->csat[0]; K.cs1 = k->csat[1]; K.cs2 = k->csat[2];
    K.T0 = k->T0; K.T1 = k->T1; K.t_cool = k->t_cool; K.kappa = k->kappa; K.cfl = k->cfl;
    K.lkg1 = std::log(K.kg1); K.lkg2 = std::log(K.kg2); K.lkb = std::log(K.kb);
    K.inv_tcool = 1.0 / K.t_cool;
    K.scheme = k->scheme;
    K.growth_form = k->growth_form;
    K.solubility_form = k->solubility_form;
    K.ea1 = k->ea[0];
    K.ea2 = k->ea[1];
    K.mW = g->d_mW;
    K.mB = g->d_mB;
    K.poly = g->d_poly;
    K.npoly = g->npoly;
    K.mbox = g->mbox;
    for (int k = 0; k < 3; ++k) { K.mlo[k] = g->mlo[k]; K.mhi[k] = g->mhi[k]; }
    g->kin = K;
    g->has_kin = true;
    if (g->plain_exec) {  // kinetics are baked into the graph's kernel arguments
        cudaGraphExecDestroy(g->plain_exec);
        g->plain_exec = nullptr;
    }
    return PBE_OK;
}


pbe_status pbe_set_closure(pbe_grid* g, const float* w, int count)
{
    if (!g || !w) return fail(PBE_EINVAL, "null argument");
    if (count != pbe::kMlpNW) return fail(PBE_EINVAL, "the closure has %d weights (got %d)", pbe::kMlpNW, count);
    for (int k = 0; k < count; ++k)
        if (!std::isfinite(w[k])) return fail(PBE_EINVAL, "non-finite closure weight %d", k);
    DeviceGuard dg(g->device);
    std::vector<__nv_bfloat16> hw;
    std::vector<float> hb;
    pbe::pack_closure(w, hw, hb);
    if (!g->d_mW) {
        if (cudaMalloc(&g->d_mW, sizeof(__nv_bfloat16) * hw.size()) != cudaSuccess ||
            cudaMalloc(&g->d_mB, sizeof(float) * hb.size()) != cudaSuccess)
            return fail(PBE_ENOMEM, "allocating the closure weights failed");
    }
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    CUDA_TRY(cudaMemcpy(g->d_mW, hw.data(), sizeof(__nv_bfloat16) * hw.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(g->d_mB, hb.data(), sizeof(float) * hb.size(), cudaMemcpyHostToDevice));
    g->kin.mW = g->d_mW;
    g->kin.mB = g->d_mB;
    // FNV-1a of the stored values: grids whose gradients are summed must agree
    unsigned long long hsh = 1469598103934665603ULL;
    auto mix = [&hsh](const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) hsh = (hsh ^ c[i]) * 1099511628211ULL;
    };
    mix(hw.data(), sizeof(__nv_bfloat16) * hw.size());
    mix(hb.data(), sizeof(float) * hb.size());
    g->mhash = hsh;
    return PBE_OK;
}

pbe_status pbe_set_growth_poly(pbe_grid* g, const double* a, int K)
{
    if (!g || !a) return fail(PBE_EINVAL, "null argument");
    if (K < 1 || K > 4096) return fail(PBE_EINVAL, "the growth polynomial has 1..4096 terms a direction (got %d)", K);
    const int n = K * g->geo.ndim;
    for (int k = 0; k < n; ++k)
        if (!std::isfinite(a[k])) return fail(PBE_EINVAL, "non-finite growth coefficient %d", k);
    DeviceGuard dg(g->device);
    if (!dg.ok) return fail(PBE_ECUDA, "cannot select device %d", g->device);
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (g->npoly != K) {
        cudaFree(g->d_poly);
        g->d_poly = nullptr;
        g->npoly = 0;
        if (cudaMalloc(&g->d_poly, sizeof(double) * n) != cudaSuccess) {
            cudaGetLastError();
            return fail(PBE_ENOMEM, "allocating %d growth coefficients failed", n);
        }
        g->npoly = K;
    }
    CUDA_TRY(cudaMemcpy(g->d_poly, a, sizeof(double) * n, cudaMemcpyHostToDevice));
    g->kin.poly = g->d_poly;
    g->kin.npoly = g->npoly;
    if (g->plain_exec) {  // the kinetics are baked into the graph's kernel arguments
        cudaGraphExecDestroy(g->plain_exec);
        g->plain_exec = nullptr;
    }
    return PBE_OK;
}

pbe_status pbe_set_closure_box(pbe_grid* g, const double* lo, const double* hi)
{
    if (!g) return fail(PBE_EINVAL, "null grid");
    if (!lo || !hi) {
        g->mbox = 0;
    } else {
        for (int k = 0; k < 3; ++k)
            if (std::isnan(lo[k]) || std::isnan(hi[k]) || !(lo[k] <= hi[k]))
                return fail(PBE_EINVAL, "closure box: lo[%d] <= hi[%d] required", k, k);
        g->mbox = 1;
        for (int k = 0; k < 3; ++k) { g->mlo[k] = lo[k]; g->mhi[k] = hi[k]; }
    }
    g->kin.mbox = g->mbox;
    for (int k = 0; k < 3; ++k) { g->kin.mlo[k] = g->mlo[k]; g->kin.mhi[k] = g->mhi[k]; }
    if (g->plain_exec) {  // the kinetics are baked into the graph's kernel arguments
        cudaGraphExecDestroy(g->plain_exec);
        g->plain_exec = nullptr;
    }
    return PBE_OK;
}

pbe_status pbe_set_state(pbe_grid* g, const double* n, double C, double t, int mem)
{
    if (!g || !n) return fail(PBE_EINVAL, "null argument");
    if (mem != PBE_MEM_HOST && mem != PBE_MEM_DEVICE) return fail(PBE_EINVAL, "bad mem flag");
    if (!std::isfinite(C) || !std::isfinite(t)) return fail(PBE_EINVAL, "non-finite C or t");
    DeviceGuard dg(g->device);
    if (!dg.ok) return fail(PBE_ECUDA, "cannot select device %d", g->device);
    CUDA_TRY(cudaMemcpyAsync(g->d_n, n, sizeof(double) * g->ncell, kind_to_device(mem), g->stream));
    CUDA_TRY(pbe::launch_set_scalars(g, C, t));
    g->C_host = C;
    g->t_host = t;
    g->has_state = true;
    return PBE_OK;
}

namespace {

// by_mass = false: scale so that sum(n) dA = total; true: so that
// rho_kv sum(x1 x2^2 n) dA (x^3 in 1-D) = total
pbe_status init_seed(pbe_grid* g, const double* mean, const double* sd, double corr, double total, bool by_mass,
                     double rho_kv, double C0)
{
    if (!g || !mean || !sd) return fail(PBE_EINVAL, "null argument");
    const int nd = g->geo.ndim;
    for (int d = 0; d < nd; ++d)
        if (!std::isfinite(mean[d]) || !(sd[d] > 0.0) || !std::isfinite(sd[d]))
            return fail(PBE_EINVAL, "seed mean must be finite and sd positive (direction %d)", d);
    if (nd == 2 && !(std::fabs(corr) < 1.0)) return fail(PBE_EINVAL, "correlation must lie in (-1, 1)");
    if (!(total > 0.0) || !std::isfinite(total)) return fail(PBE_EINVAL, "the seed total must be positive and finite");
    if (by_mass && (!(rho_kv > 0.0) || !std::isfinite(rho_kv))) return fail(PBE_EINVAL, "rho_kv must be positive");
    if (!std::isfinite(C0)) return fail(PBE_EINVAL, "non-finite C0");
    DeviceGuard dg(g->device);
    if (!dg.ok) return fail(PBE_ECUDA, "cannot select device %d", g->device);
    g->has_state = false;
    CUDA_TRY(pbe::launch_seed_pdf(g, mean, sd, nd == 2 ? corr : 0.0, g->d_mom));
    CUDA_TRY(cudaMemcpyAsync(g->h_stage, g->d_mom, 2 * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    const double sum = by_mass ? rho_kv * g->h_stage[1] : g->h_stage[0];
    if (!(sum > 0.0) || !std::isfinite(sum))
        return fail(PBE_EINVAL, "the seed has no mass on the grid (its density underflows at every cell centre)");
    const double scale = nd == 1 ? total / (sum * g->geo.d1) : total / (sum * g->geo.d1 * g->geo.d2);
    CUDA_TRY(pbe::launch_scale(g, scale));
    CUDA_TRY(pbe::launch_set_scalars(g, C0, 0.0));
    g->C_host = C0;
    g->t_host = 0.0;
    g->has_state = true;
    return PBE_OK;
}

}  // namespace

pbe_status pbe_init_seed_gaussian(pbe_grid* g, const double* mean, const double* sd, double corr,
                                  double total_number, double C0)
{
    return init_seed(g, mean, sd, corr, total_number, false, 0.0, C0);
}

pbe_status pbe_init_seed_gaussian_mass(pbe_grid* g, const double* mean, const double* sd, double corr,
                                       double seed_mass, double rho_kv, double C0)
{
    return init_seed(g, mean, sd, corr, seed_mass, true, rho_kv, C0);
}

pbe_status pbe_get_state(pbe_grid* g, double* n, double* C, double* t, int mem)
{
    if (!g) return fail(PBE_EINVAL, "null grid");
    if (!g->has_state) return fail(PBE_ESTATE, "no state set");
    DeviceGuard dg(g->device);
    if (n) CUDA_TRY(cudaMemcpyAsync(n, g->d_n, sizeof(double) * g->ncell, kind_from_device(mem), g->stream));
    CUDA_TRY(cudaMemcpyAsync(g->h_S, g->d_S, sizeof(Scal), cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (C) *C = g->h_S->C;
    if (t) *t = g->h_S->t;
    return PBE_OK;
}

pbe_status pbe_solve(pbe_grid* g, const double* t_out, int n_out, double* rows, int mem, int64_t* steps)
{
    if (!g || !t_out || !rows) return fail(PBE_EINVAL, "null argument");
    if (n_out < 1) return fail(PBE_EINVAL, "n_out must be >= 1");
    if (mem != PBE_MEM_HOST && mem != PBE_MEM_DEVICE) return fail(PBE_EINVAL, "bad mem flag");
    if (!g->has_kin || !g->has_state) return fail(PBE_ESTATE, "set kinetics and state before solving");
    if (!std::isfinite(t_out[0]) || t_out[0] < g->t_host)
        return fail(PBE_EINVAL, "t_out[0] = %g precedes the current time %g", t_out[0], g->t_host);
    for (int j = 1; j < n_out; ++j)
        if (!(t_out[j] > t_out[j - 1]) || !std::isfinite(t_out[j]))
            return fail(PBE_EINVAL, "t_out must be strictly increasing and finite (index %d)", j);
    DeviceGuard dg(g->device);
    if (!dg.ok) return fail(PBE_ECUDA, "cannot select device %d", g->device);
    pbe_status st = pbe::prepare_tout(g, t_out, n_out);
    if (st) return st;
    g->kernel_ms = -1.0;
    st = run_solve(g, n_out);
    if (st) return st;
    CUDA_TRY(cudaMemcpyAsync(rows, g->d_rows, sizeof(double) * n_out * ncol_of(g), kind_from_device(mem), g->stream));
    st = finish_call(g);
    if (steps) *steps = g->h_S->steps;
    if (g->timing) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, g->ev_k0, g->ev_k1) == cudaSuccess) g->kernel_ms = ms;
    }
    return st;
}

pbe_status pbe_set_timing(pbe_grid* g, int enable)
{
    if (!g) return fail(PBE_EINVAL, "null grid");
    DeviceGuard dg(g->device);
    if (!dg.ok) return fail(PBE_ECUDA, "cannot select device %d", g->device);
    if (enable && !g->ev_k0) {
        CUDA_TRY(cudaEventCreate(&g->ev_k0));
        CUDA_TRY(cudaEventCreate(&g->ev_k1));
    }
    g->timing = enable != 0;
    g->kernel_ms = -1.0;
    return PBE_OK;
}

pbe_status pbe_kernel_time(pbe_grid* g, double* ms)
{
    if (!g || !ms) return fail(PBE_EINVAL, "null argument");
    *ms = g->kernel_ms;
    return PBE_OK;
}

pbe_status pbe_step(pbe_grid* g, double t_limit, double* dt_taken)
{
    if (!g) return fail(PBE_EINVAL, "null grid");
    if (!g->has_kin || !g->has_state) return fail(PBE_ESTATE, "set kinetics and state before stepping");
    if (!(t_limit > g->t_host) || !std::isfinite(t_limit))
        return fail(PBE_EINVAL, "t_limit = %g must exceed the current time %g", t_limit, g->t_host);
    DeviceGuard dg(g->device);
    if (!dg.ok) return fail(PBE_ECUDA, "cannot select device %d", g->device);
    pbe_status st = ensure_tout_capacity(g, 1);
    if (st) return st;
    g->h_stage[0] = t_limit;
    CUDA_TRY(cudaMemcpyAsync(g->d_tout, g->h_stage, sizeof(double), cudaMemcpyHostToDevice, g->stream));
    g->tout_valid_n = 0;
    CUDA_TRY(pbe::launch_prologue(g, 1, 1, nullptr));
    CUDA_TRY(pbe::launch_plain_step(g, false, 0));
    CUDA_TRY(pbe::launch_paper_finish(g));
    st = finish_call(g);
    if (dt_taken) *dt_taken = g->h_S->last_dt;
    if (st == PBE_ETIMEOUT) st = PBE_OK;  // the one-step budget is the point of this call
    return st;
}

pbe_status pbe_moments(pbe_grid* g, double* mu, int mem)
{
    if (!g || !mu) return fail(PBE_EINVAL, "null argument");
    if (!g->has_state) return fail(PBE_ESTATE, "no state set");
    DeviceGuard dg(g->device);
    CUDA_TRY(pbe::launch_prologue(g, 0, 0, g->d_mom));
    int nm = g->geo.ndim == 1 ? 4 : 10;
    CUDA_TRY(cudaMemcpyAsync(mu, g->d_mom, sizeof(double) * nm, kind_from_device(mem), g->stream));
    if (mem == PBE_MEM_HOST) CUDA_TRY(cudaStreamSynchronize(g->stream));
    return PBE_OK;
}

}  // extern "C"

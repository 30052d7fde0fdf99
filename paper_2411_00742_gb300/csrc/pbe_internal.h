// Host-side state of a grid and the launchers of each execution path.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "pbe.h"
#include "pbe_device.cuh"

namespace pbe {
struct AdjWork;   // buffers of the persistent adjoint (pbe_adjoint_fused.cu)
}

struct pbe_grid {
    int device;
    pbe::Geom geo;
    pbe::Kin kin;
    bool has_kin, has_state;
    int path;
    cudaStream_t stream;
    long long max_steps;
    size_t ncell;
    double* d_n;        // state n
    double* d_n1;       // stage-1 buffer
    pbe::Scal* d_S;     // scalars
    double* d_part;     // block partials [max_blocks][kMaxMom]
    double* d_mom;      // moments read-out (kMaxMom doubles)
    unsigned int* d_bar; // fused path: 512 bytes of barrier accumulators (two 64-bit words, 128 B apart)
    int max_blocks;
    int sms;            // multiprocessors of the grid's device
    int window_mode;    // 2-D plain stages in the register-window kernel: -1 auto, 0 never, 1 always
    int block_limit;    // most blocks of the fused path's persistent launches (0: no limit)
    // fused path launch configuration, fixed per grid (computed at the first fused solve)
    const void* fused_fn;
    int fused_blocks, fused_ntiles, fused_tiles_x, fused_ti;
    size_t fused_dyn;   // dynamic shared memory of that kernel
    double* d_tout;     // output times (capacity tout_cap)
    double* d_rows;     // output rows (capacity tout_cap rows of 12)
    double* d_rowpart;  // fused path: per-row, per-block moment partials (tout_cap x max_blocks/2 x 10)
    int tout_cap;
    double* h_tout;     // pinned copy of the output times last sent to d_tout (capacity tout_cap)
    int tout_valid_n;   // number of entries of d_tout equal to h_tout (0: none)
    pbe::Scal* h_S;     // pinned copy of the scalars
    double* h_stage;    // pinned staging for small host<->device copies (64 doubles)
    // plain-path graph: prologue + while-loop over the two stage kernels
    cudaGraphExec_t plain_exec;
    bool plain_graph_failed;
    double C_host, t_host;  // host mirror of the scalar state after the last synchronizing call
    long long wait_cycles;  // device-wide wait limit of the fused path (-1: default ~1 s)
    __nv_bfloat16* d_mW;    // learned closure weights (bf16) and biases (fp32)
    float* d_mB;
    double* d_poly;         // polynomial growth law (Eq. 6): ndim x npoly coefficients
    int npoly;
    unsigned long long mhash;  // learned closure: hash of the stored weights (grids that share them agree)
    int mbox;               // learned closure: training box of its inputs (pbe_set_closure_box)
    double mlo[3], mhi[3];
    // optional device timing of the launch that advances the state in pbe_solve
    bool timing;
    cudaEvent_t ev_k0, ev_k1;
    double kernel_ms;       // duration of that launch in the last solve (-1: none)
    pbe::AdjWork* adjw;     // persistent adjoint: checkpoint store and work buffers, kept between calls
};

namespace pbe {

// one instance of a batch (device descriptor)
struct BatchInst {
    Kin K;
    Geom g;
    long long offset;   // first cell in the packed state
    int rows;           // ceil(N / 32)
    int pad;
};

// number of block partial slots the plain kernels of this grid use
int plain_max_blocks(const Geom& g);

// Plain path (pbe_plain.cu)
cudaError_t launch_prologue(pbe_grid* g, int n_out, long long max_steps, double* mom_out);
cudaError_t launch_plain_step(pbe_grid* g, bool use_cond, cudaGraphConditionalHandle h);
cudaError_t launch_plain_stage(pbe_grid* g, int stage);
cudaError_t launch_set_scalars(pbe_grid* g, double C, double t);

// Plain path, large 2-D grids (pbe_window.cu): one SSP-RK2 stage per kernel
// in the register-window layout; by default used when it gives at least one
// block per SM (pbe_set_window)
bool use_window2d(const pbe_grid* g);
cudaError_t window_setup();   // shared-memory limit of the kernels, on the current device
cudaError_t launch_window_stage2d(pbe_grid* g, int stage, bool use_cond, cudaGraphConditionalHandle h);
// Fused path, the same grids (pbe_window.cu): the persistent window kernel
// (k_fused's parameters) and its launch shape
struct FusedWinCfg {
    const void* fn;
    size_t dyn;
    int G, ntiles, tiles_x, ti;
};
cudaError_t fused_window_config(const Geom& g, int sms, int max_blocks, FusedWinCfg* c);
// unscaled Gaussian density at the cell centres into d_n; total_dev[0] = its sum,
// total_dev[1] = its sum weighted by x^3 (1-D) or x1 x2^2 (2-D)
cudaError_t launch_seed_pdf(pbe_grid* g, const double* mean, const double* sd, double corr, double* total_dev);
cudaError_t launch_scale(pbe_grid* g, double a);   // d_n *= a

// The paper's split scheme in 2-D (pbe_paper.cu): one kernel per step, the
// state alternating between d_n and d_n1; launch_paper_finish puts it back
// in d_n after the last step (no launch for other schemes).
cudaError_t launch_paper_step2d(pbe_grid* g, bool use_cond, cudaGraphConditionalHandle h);
cudaError_t launch_paper_finish(pbe_grid* g);
int paper_blocks2d(const Geom& g);

// Value checks of a pbe_kinetics shared by every entry point that takes one
// (pbe_api.cu): PBE_OK, or PBE_EINVAL with the error message set.
pbe_status check_kinetic_values(const pbe_kinetics* k);

// The learned closure's flat weights (W1, b1, W2, b2, W3, b3; kMlpNW floats)
// as the kernels store them: bf16 matrices and fp32 biases (pbe_api.cu).
void pack_closure(const float* w, std::vector<__nv_bfloat16>& hw, std::vector<float>& hb);

// Output times of a solve on the device (d_tout, capacity grown as needed;
// the copy is skipped when they equal the last ones sent) (pbe_api.cu).
pbe_status prepare_tout(pbe_grid* g, const double* t_out, int n_out);

// Persistent adjoint (pbe_adjoint_fused.cu): pbe_vjp on the fused path, with
// the arguments pbe_vjp has checked; adjoint_work_free releases its buffers.
pbe_status vjp_persistent(pbe_grid* g, const double* t_out, int n_out, const double* seeds, int seeds_mem, int K,
                          double* dL_dtheta, double* dL_dn0, double* dL_dC0, double* rows, int mem,
                          double* dL_dweights);
void adjoint_work_free(pbe_grid* g);
// A fused-path solve with the learned closure: the persistent kernel's forward
// pass (per-stage mu0 sums for the closure's moment-ratio input).
cudaError_t launch_solve_persistent(pbe_grid* g, int n_out);

// The learned closure's weight gradient over recorded evaluations
// (pbe_mlp_grad.cu): rows of (x0, x1, x2, lo0, lo1, lo2) floats, tensor-core
// contractions; `part` is a workspace of mlp_grad_part_floats() floats.
int mlp_grad_part_floats();
cudaError_t launch_mlp_grad(const float* rows, long long R, const __nv_bfloat16* mW, const float* mB, float* part,
                            double* dW, cudaStream_t st);

// Fused path (pbe_fused.cu)
cudaError_t launch_fused_solve(pbe_grid* g, int n_out);
bool fused_supported(const pbe_grid* g);

}  // namespace pbe

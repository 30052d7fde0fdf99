// Fused path for one grid: a single persistent cooperative launch runs the
// whole solve.  Each block owns a fixed set of tiles; the two stages of every
// step are separated by a device-wide barrier.  After each barrier the block
// splits: warp 0 sums the per-block moment partials in a fixed order and
// advances the block's private copy of the scalar chain (solute balance,
// kinetics, CFL step - identical in every block), while the other warps
// already load the next stage's input tile and compute its face values,
// which do not depend on the kinetics.  Face quotients use the
// Newton-Raphson form (half_psi_fast).
//
// Every wait is bounded: a barrier that does not complete within about one
// second sets PBE_ETIMEOUT and the kernel returns.
#include <type_traits>

#include "pbe_internal.h"
#include "pbe_tiles.cuh"

namespace pbe {

constexpr int kFNT = 256;     // threads per block
constexpr int kFT1 = 1024;    // 1-D tile
constexpr int kFTI = 8;       // 2-D tile rows
constexpr int kFTJ = 32;      // 2-D tile columns
constexpr long long kBarrierCycles = 2000000000LL;  // ~1 s at 2 GHz

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned int* p, unsigned int v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Device-wide barrier over gridDim.x co-resident blocks (cooperative launch).
// bar[0] counts arrivals, bar[1] is the generation.  Returns false on timeout.
__device__ bool grid_barrier(unsigned int* bar, unsigned int& gen, int* fail_sh)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int target = gen + 1u;
        int ok = 1;
        __threadfence();
        const unsigned int arrived = atomicAdd(&bar[0], 1u);
        if (arrived == gridDim.x - 1u) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            st_release(&bar[1], target);
        } else {
            const long long t0 = clock64();
            unsigned int polls = 0;
            while (ld_acquire(&bar[1]) != target) {
                if (++polls > 64u) {
                    if (clock64() - t0 > kBarrierCycles) { ok = 0; break; }
                    __nanosleep(20);
                }
            }
        }
        __threadfence();
        gen = target;
        *fail_sh = !ok;
    }
    __syncthreads();
    return *fail_sh == 0;
}

// Sum of one moment slot over all blocks' partials, by one warp, in a fixed
// order: lane l sums blocks l, l+32, ... as a balanced tree per chunk of 16,
// then a butterfly over the lanes (every lane ends with the same value).
__device__ __forceinline__ double warp_sum_partials(const double* part, int G, int slot)
{
    const int lane = threadIdx.x & 31;
    double acc = 0.0;
    for (int base = 0; base < G; base += 32 * 16) {
        double v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int b = base + lane + 32 * k;
            v[k] = b < G ? __ldcg(part + (size_t)b * kMaxMom + slot) : 0.0;
        }
#pragma unroll
        for (int w = 8; w > 0; w >>= 1)
#pragma unroll
            for (int k = 0; k < w; ++k) v[k] += v[k + w];
        acc += v[0];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

struct GroupSync {  // named barrier over warps 1..7
    __device__ __forceinline__ void operator()() const { asm volatile("bar.sync 1, %0;" ::"r"(kFNT - 32) : "memory"); }
};
struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

template <int NDIM>
struct FusedSmem;
template <>
struct FusedSmem<1> {
    double tile[kFT1 + 3];
    double h[kFT1 + 1];
};
template <>
struct FusedSmem<2> {
    Tile2DSmem<kFTI, kFTJ> t;
};

template <int NDIM>
__device__ __forceinline__ void tile_origin(int t, int tiles_x, int& i0, int& j0)
{
    if (NDIM == 1) { i0 = t * kFT1; j0 = 0; }
    else { i0 = (t / tiles_x) * kFTI; j0 = (t % tiles_x) * kFTJ; }
}

// faces of tile t of `in` on threads [tid, tid+nthr) of the block
template <int NDIM, class Sync>
__device__ __forceinline__ void fused_faces(const double* in, int t, int tiles_x, const Geom& g, FusedSmem<NDIM>& sm,
                                            int tid, int nthr, Sync sync)
{
    int i0, j0;
    tile_origin<NDIM>(t, tiles_x, i0, j0);
    if constexpr (NDIM == 1) faces1d<true, true, kFT1>(in, i0, g, sm.tile, sm.h, tid, nthr, sync);
    else faces2d<true, true, kFTI, kFTJ>(in, i0, j0, g, sm.t, tid, nthr, sync);
}

template <int STAGE, int NDIM, int NM>
__device__ __forceinline__ void fused_cells(const double* old, double* out, int t, int tiles_x, const Geom& g,
                                            const StageCoef& sc, double (&m)[NM], const FusedSmem<NDIM>& sm)
{
    int i0, j0;
    tile_origin<NDIM>(t, tiles_x, i0, j0);
    if constexpr (NDIM == 1) cells1d<STAGE, kFT1, kFNT>(old, out, i0, g, sc, m, sm.tile, sm.h);
    else cells2d<STAGE, kFTI, kFTJ, kFNT>(old, out, i0, j0, g, sc, m, sm.t);
}

// One stage over all tiles of this block; the first tile's faces are already
// in shared memory.  in: stage input, old/out: see tile1d/tile2d.
template <int STAGE, int NDIM, int NM>
__device__ __forceinline__ void fused_stage(const double* in, const double* old, double* out, int ntiles, int tiles_x,
                                            const Geom& g, const StageCoef& sc, double (&m)[NM], FusedSmem<NDIM>& sm)
{
    const int G = gridDim.x;
    for (int t = blockIdx.x; t < ntiles; t += G) {
        if (t != (int)blockIdx.x) {
            fused_faces<NDIM>(in, t, tiles_x, g, sm, threadIdx.x, kFNT, BlockSync());
            __syncthreads();
        }
        fused_cells<STAGE, NDIM, NM>(old, out, t, tiles_x, g, sc, m, sm);
        __syncthreads();
    }
}

template <int NDIM>
__global__ void __launch_bounds__(kFNT) k_fused(double* n, double* n1, Scal* S, Kin K, Geom g, double* part,
                                                const double* t_out, double* rows, unsigned int* bar, int ntiles,
                                                int tiles_x)
{
    constexpr int NM = NDIM == 1 ? 4 : 10;
    constexpr int VIDX = NDIM == 1 ? 3 : 8;
    __shared__ Scal s;
    __shared__ double sh[kFNT / 32 * NM];
    __shared__ double msum[NM];
    __shared__ int fail;
    __shared__ FusedSmem<NDIM> sm;
    if (threadIdx.x == 0) s = *S;
    __syncthreads();
    if (s.done) return;
    const int G = gridDim.x;
    const int warp = threadIdx.x >> 5;
    double* part1 = part;                        // stage-1 partials [G][kMaxMom]
    double* part2 = part + (size_t)G * kMaxMom;  // stage-2 partials
    double* my_rows = blockIdx.x == 0 ? rows : nullptr;
    unsigned int gen = 0;

    fused_faces<NDIM>(n, blockIdx.x, tiles_x, g, sm, threadIdx.x, kFNT, BlockSync());
    __syncthreads();
    for (;;) {
        // ---- stage 1: n1 = n + dt L(n) ----
        {
            const StageCoef sc = stage_coef<1>(s, g);
            double m[NM];
#pragma unroll
            for (int k = 0; k < NM; ++k) m[k] = 0.0;
            fused_stage<1, NDIM, NM>(n, n, n1, ntiles, tiles_x, g, sc, m, sm);
            double v[1] = {m[VIDX]};
            block_sum<kFNT, 1>(v, sh);
            if (threadIdx.x == 0) part1[(size_t)blockIdx.x * kMaxMom + VIDX] = v[0];
            if (!grid_barrier(bar, gen, &fail)) break;
            if (warp == 0) {
                const double V1 = warp_sum_partials(part1, G, VIDX);
                finish_stage1_warp(&s, K, V1);
            } else {
                fused_faces<NDIM>(n1, blockIdx.x, tiles_x, g, sm, threadIdx.x - 32, kFNT - 32, GroupSync());
            }
            __syncthreads();
            if (s.done) break;
        }
        // ---- stage 2: n = n/2 + (n1 + dt L(n1))/2 ----
        {
            const StageCoef sc = stage_coef<2>(s, g);
            double m[NM];
#pragma unroll
            for (int k = 0; k < NM; ++k) m[k] = 0.0;
            fused_stage<2, NDIM, NM>(n1, n, n, ntiles, tiles_x, g, sc, m, sm);
            if (sc.moms) {
                block_sum<kFNT, NM>(m, sh);
                if (threadIdx.x == 0)
                    for (int k = 0; k < NM; ++k) part2[(size_t)blockIdx.x * kMaxMom + k] = m[k];
            } else {
                double v[1] = {m[VIDX]};
                block_sum<kFNT, 1>(v, sh);
                if (threadIdx.x == 0) part2[(size_t)blockIdx.x * kMaxMom + VIDX] = v[0];
            }
            if (!grid_barrier(bar, gen, &fail)) break;
            if (warp == 0) {
                if (sc.moms) {
                    for (int k = 0; k < NM; ++k) {
                        const double tot = warp_sum_partials(part2, G, k);
                        if (threadIdx.x == 0) msum[k] = tot;
                    }
                } else {
                    const double tot = warp_sum_partials(part2, G, VIDX);
                    if (threadIdx.x == 0) msum[VIDX] = tot;
                }
                __syncwarp();
                finish_stage2_warp(&s, K, g, t_out, my_rows, msum, NM, VIDX);
            } else {
                fused_faces<NDIM>(n, blockIdx.x, tiles_x, g, sm, threadIdx.x - 32, kFNT - 32, GroupSync());
            }
            __syncthreads();
            if (s.done) break;
        }
    }
    if (threadIdx.x == 0 && fail) {
        S->status = PBE_ETIMEOUT;
        S->done = 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && !fail) {
        s.counter = 0u;
        *S = s;
    }
}

static int fused_tiles(const Geom& g, int* tiles_x)
{
    if (g.ndim == 1) {
        *tiles_x = 1;
        return (g.N1 + kFT1 - 1) / kFT1;
    }
    *tiles_x = (g.N2 + kFTJ - 1) / kFTJ;
    return *tiles_x * ((g.N1 + kFTI - 1) / kFTI);
}

bool fused_supported(const pbe_grid* g) { return g->d_bar != nullptr; }

cudaError_t launch_fused_solve(pbe_grid* g, int n_out)
{
    (void)n_out;
    int tiles_x;
    const int ntiles = fused_tiles(g->geo, &tiles_x);
    const void* fn = g->geo.ndim == 1 ? (const void*)k_fused<1> : (const void*)k_fused<2>;
    int occ = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kFNT, 0);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e != cudaSuccess) return e;
    int G = ntiles;
    if (G > occ * sms) G = occ * sms;
    if (2 * G > g->max_blocks) G = g->max_blocks / 2;
    if (G < 1) G = 1;
    e = cudaMemsetAsync(g->d_bar, 0, 2 * sizeof(unsigned int), g->stream);
    if (e != cudaSuccess) return e;
    void* args[] = {&g->d_n, &g->d_n1, &g->d_S, &g->kin, &g->geo, &g->d_part, &g->d_tout, &g->d_rows,
                    &g->d_bar, (void*)&ntiles, &tiles_x};
    return cudaLaunchCooperativeKernel(fn, G, kFNT, args, 0, g->stream);
}

}  // namespace pbe
